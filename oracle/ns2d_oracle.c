/*
 * ns2d_oracle.c -- plain, slow, FP64 CPU oracle for the EnVar open-cavity hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py may load this library.  The product
 * path (paper_2605_23812_gb300) never links, imports or calls it, and shares no
 * code, header, table or helper with it.
 *
 * What it computes, in the paper's terms (arXiv 2605.23812):
 *   - the forced incompressible Navier-Stokes equations, Sec. 2, Eq. (forced_NS),
 *     in the semi-discrete form L dq/dt + N(q) = P f of Eq. (discrete_NS), here
 *     discretised on a staggered MAC grid with explicit Adams-Bashforth-2 for
 *     advection + diffusion + forcing and an incremental pressure projection
 *     (the paper's own FEM/BDF2 solver, Sec. 4.4, is prior art, not reproduced);
 *   - the observation cost of Sec. 4.1, Eq. (specific_cost_function), as sensor
 *     fluctuations u' = u - mean(u) at x = 1/5..4/5, y = 0 (SENSORS), and the
 *     domain-integrated fluctuation energy of Eq. (kinenergy) normalised by the
 *     number of window samples (DOMAIN);
 *   - the ensemble representation f = f_e + E w, Eq. (ensemble_representation),
 *     with columns of E drawn from N(0, B) for the Gaussian kernel B of
 *     Eq. (covarianceB) with c_xy = infinity (Sec. 3.3.2 / Sec. 4.2);
 *   - the finite-difference ensemble sensitivities of Eq. (fdapprox) and the
 *     EnVar gradient of Eq. (gradient_EnVar) in w-space (prior term
 *     (N-1) w from Eq. (J_w)): the scalar-anomaly form from the member costs,
 *     and the explicit contraction Y^T (Hq_0 - y) on the sensor series and on
 *     the domain observation vector;
 *   - the weight update of Sec. 3.3.1 with the prior-Hessian step.
 *
 * Parity status of each function is listed with the function.  Every function
 * below is pinned by a -m "not gpu" test except where the header says
 * "parity unpinned".
 *
 * Numerical choices (the paper is silent on all of them, so each is a reading
 * made for this solver):
 *   * fluid cell  <=> its centre has y > 0, or 0 < x < 1 (open cavity, staircase);
 *   * u (v) face is an unknown iff both adjacent cells are fluid; a face with
 *     one fluid neighbour is a wall (normal velocity 0); a face with no fluid
 *     neighbour takes, inside a stencil, the mirror value of the fluid-side face
 *     (no-slip by reflection about the wall);
 *   * inlet u = erf(y / delta), v = 0 by reflection; top free slip; bottom
 *     no-slip; outlet: convective u_b^{n+1} = u_b^n - dt Uc (u_b^n - u_{nx-1}^n)/dx,
 *     then a uniform additive shift so outflow flux == inflow flux; v at the
 *     outlet has zero normal gradient;
 *   * first step forward Euler, then AB2; incremental projection with the
 *     pressure increment solved by Jacobi-preconditioned CG on the masked
 *     Neumann Laplacian, mean zero over fluid cells.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_VERSION 1

/* ------------------------------------------------------------------------- */
/* Parameters (mirrored by a ctypes Structure in oracle/__init__.py).          */
/* ------------------------------------------------------------------------- */
typedef struct {
    int nx, ny;
    double x0, x1, y0, y1;
    double Re;
    double dt;
    int bc_x;        /* 0: inlet (left) / convective outlet (right); 1: periodic */
    int bc_y;        /* 0: no-slip bottom, free-slip top; 1: periodic; 2: no-slip both */
    int geometry;    /* 0: open cavity; 1: all fluid; 2: fluid iff ch_lo<yc<ch_hi; 3: fluid iff ch_lo<xc<ch_hi */
    int advection;   /* 1: include the advection term; 0: Stokes flow */
    double inlet_delta;  /* inlet profile erf(y / inlet_delta) */
    double conv_speed;   /* convective outflow speed Uc */
    double cg_rtol;      /* CG stops when ||r||_2 <= cg_rtol * ||rhs||_2 */
    int cg_maxit;
    double ch_lo, ch_hi; /* channel bounds for geometry 2 / 3 */
    int lip_slip;        /* 1: a solid face under a fluid face (a lower wall) whose x lies outside
                            [slip_lo, slip_hi] reflects evenly (free slip) instead of oddly (no slip):
                            the slip segments of the paper's lower wall (Sec. 4.4) */
    double slip_lo, slip_hi;
} orc_params;

enum { FK_WALL = 0, FK_UNKNOWN = 1, FK_INLET = 2, FK_OUTLET = 3, FK_SOLID = 4, FK_COPY = 5 };

typedef struct {
    orc_params P;
    int nx, ny;
    double dx, dy, nu;
    unsigned char *F;          /* fluid cells [j*nx+i] */
    unsigned char *uk, *vk;    /* face kinds   u: [j*(nx+1)+i]  v: [j*nx+i] */
    double *u, *v, *p;         /* state (compact) */
    double *Ru, *Rv;           /* previous explicit right-hand side (AB2) */
    double *fu, *fv;           /* face forcing */
    double *Ug, *Vg;           /* ghost-padded copies of u, v */
    double *us, *vs;           /* predictor */
    double *rhs, *dp, *cr, *cz, *cp, *cq, *diag;
    double *ub_next;
    int *nbE, *nbW, *nbN, *nbS;/* Poisson neighbour cell index, or -1 if the face between is closed */
    long nstep;                /* completed steps */
    int last_cg_iters;
    double last_cg_relres;
} orc_sim;

/* index helpers (compact arrays) */
#define IU(s, i, j) ((size_t)(j) * (size_t)((s)->nx + 1) + (size_t)(i))
#define IV(s, i, j) ((size_t)(j) * (size_t)((s)->nx) + (size_t)(i))
#define IC(s, i, j) ((size_t)(j) * (size_t)((s)->nx) + (size_t)(i))
/* ghost-padded: Ug has i in [-1, nx+1], j in [-1, ny]; Vg has i in [-1, nx], j in [-1, ny+1] */
#define UG(s, i, j) ((s)->Ug[(size_t)((j) + 1) * (size_t)((s)->nx + 3) + (size_t)((i) + 1)])
#define VG(s, i, j) ((s)->Vg[(size_t)((j) + 1) * (size_t)((s)->nx + 2) + (size_t)((i) + 1)])

static int wrap(int i, int n) { return ((i % n) + n) % n; }

double orc_cell_xc(const orc_params *P, int i) { return P->x0 + ((double)i + 0.5) * ((P->x1 - P->x0) / P->nx); }
double orc_cell_yc(const orc_params *P, int j) { return P->y0 + ((double)j + 0.5) * ((P->y1 - P->y0) / P->ny); }

int orc_version(void) { return ORC_VERSION; }

/* Fluid mask.  geometry 0 is the open cavity of Fig. 1 / Table 1 on the box
 * given by the parameters: fluid above y = 0, and inside the cavity 0 < x < 1. */
void orc_fluid_mask(const orc_params *P, unsigned char *F)
{
    for (int j = 0; j < P->ny; ++j)
        for (int i = 0; i < P->nx; ++i) {
            double xc = orc_cell_xc(P, i), yc = orc_cell_yc(P, j);
            int f = 1;
            if (P->geometry == 0) f = (yc > 0.0) || (xc > 0.0 && xc < 1.0);
            else if (P->geometry == 2) f = (yc > P->ch_lo) && (yc < P->ch_hi);
            else if (P->geometry == 3) f = (xc > P->ch_lo) && (xc < P->ch_hi);
            F[(size_t)j * P->nx + i] = (unsigned char)f;
        }
}

static int fl(const orc_sim *s, int i, int j)
{
    if (s->P.bc_x == 1) i = wrap(i, s->nx);
    if (s->P.bc_y == 1) j = wrap(j, s->ny);
    if (i < 0 || i >= s->nx || j < 0 || j >= s->ny) return 0;
    return s->F[IC(s, i, j)];
}

static double inlet_profile(const orc_sim *s, int j)
{
    double y = orc_cell_yc(&s->P, j);
    return erf(y / s->P.inlet_delta);
}

static void classify_faces(orc_sim *s)
{
    int nx = s->nx, ny = s->ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            unsigned char k;
            if (s->P.bc_x == 1) {
                if (i == nx) k = FK_COPY;
                else {
                    int a = fl(s, i - 1, j), b = fl(s, i, j);
                    k = (a && b) ? FK_UNKNOWN : ((a || b) ? FK_WALL : FK_SOLID);
                }
            } else if (i == 0) {
                k = fl(s, 0, j) ? FK_INLET : FK_WALL;
            } else if (i == nx) {
                k = fl(s, nx - 1, j) ? FK_OUTLET : FK_WALL;
            } else {
                int a = fl(s, i - 1, j), b = fl(s, i, j);
                k = (a && b) ? FK_UNKNOWN : ((a || b) ? FK_WALL : FK_SOLID);
            }
            s->uk[IU(s, i, j)] = k;
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            unsigned char k;
            if (s->P.bc_y == 1) {
                if (j == ny) k = FK_COPY;
                else {
                    int a = fl(s, i, j - 1), b = fl(s, i, j);
                    k = (a && b) ? FK_UNKNOWN : ((a || b) ? FK_WALL : FK_SOLID);
                }
            } else if (j == 0 || j == ny) {
                k = FK_WALL;
            } else {
                int a = fl(s, i, j - 1), b = fl(s, i, j);
                k = (a && b) ? FK_UNKNOWN : ((a || b) ? FK_WALL : FK_SOLID);
            }
            s->vk[IV(s, i, j)] = k;
        }
}

static void *xcalloc(size_t n, size_t sz)
{
    void *p = calloc(n ? n : 1, sz);
    if (!p) { fprintf(stderr, "oracle: out of memory\n"); abort(); }
    return p;
}

static int conn_e(const orc_sim *s, int i, int j);
static int conn_w(const orc_sim *s, int i, int j);
static int conn_n(const orc_sim *s, int i, int j);
static int conn_s(const orc_sim *s, int i, int j);

static void build_neighbours(orc_sim *s)
{
    int nx = s->nx, ny = s->ny;
    size_t nc = (size_t)nx * ny;
    s->nbE = (int *)xcalloc(nc, sizeof(int)); s->nbW = (int *)xcalloc(nc, sizeof(int));
    s->nbN = (int *)xcalloc(nc, sizeof(int)); s->nbS = (int *)xcalloc(nc, sizeof(int));
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = IC(s, i, j);
            int f = s->F[k];
            s->nbE[k] = (f && conn_e(s, i, j)) ? (int)IC(s, wrap(i + 1, nx), j) : -1;
            s->nbW[k] = (f && conn_w(s, i, j)) ? (int)IC(s, wrap(i - 1, nx), j) : -1;
            s->nbN[k] = (f && conn_n(s, i, j)) ? (int)IC(s, i, wrap(j + 1, ny)) : -1;
            s->nbS[k] = (f && conn_s(s, i, j)) ? (int)IC(s, i, wrap(j - 1, ny)) : -1;
        }
}

orc_sim *orc_create(const orc_params *P)
{
    if (P->nx < 2 || P->ny < 2) return NULL;
    orc_sim *s = (orc_sim *)xcalloc(1, sizeof(orc_sim));
    s->P = *P;
    s->nx = P->nx; s->ny = P->ny;
    s->dx = (P->x1 - P->x0) / P->nx;
    s->dy = (P->y1 - P->y0) / P->ny;
    s->nu = 1.0 / P->Re;
    size_t nc = (size_t)s->nx * s->ny, nu_ = (size_t)(s->nx + 1) * s->ny, nv_ = (size_t)s->nx * (s->ny + 1);
    s->F = (unsigned char *)xcalloc(nc, 1);
    s->uk = (unsigned char *)xcalloc(nu_, 1);
    s->vk = (unsigned char *)xcalloc(nv_, 1);
    s->u = (double *)xcalloc(nu_, sizeof(double));
    s->v = (double *)xcalloc(nv_, sizeof(double));
    s->p = (double *)xcalloc(nc, sizeof(double));
    s->Ru = (double *)xcalloc(nu_, sizeof(double));
    s->Rv = (double *)xcalloc(nv_, sizeof(double));
    s->fu = (double *)xcalloc(nu_, sizeof(double));
    s->fv = (double *)xcalloc(nv_, sizeof(double));
    s->us = (double *)xcalloc(nu_, sizeof(double));
    s->vs = (double *)xcalloc(nv_, sizeof(double));
    s->Ug = (double *)xcalloc((size_t)(s->nx + 3) * (s->ny + 2), sizeof(double));
    s->Vg = (double *)xcalloc((size_t)(s->nx + 2) * (s->ny + 3), sizeof(double));
    s->rhs = (double *)xcalloc(nc, sizeof(double));
    s->dp = (double *)xcalloc(nc, sizeof(double));
    s->cr = (double *)xcalloc(nc, sizeof(double));
    s->cz = (double *)xcalloc(nc, sizeof(double));
    s->cp = (double *)xcalloc(nc, sizeof(double));
    s->cq = (double *)xcalloc(nc, sizeof(double));
    s->diag = (double *)xcalloc(nc, sizeof(double));
    s->ub_next = (double *)xcalloc((size_t)s->ny, sizeof(double));
    orc_fluid_mask(P, s->F);
    classify_faces(s);
    build_neighbours(s);
    return s;
}

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    free(s->F); free(s->uk); free(s->vk); free(s->u); free(s->v); free(s->p);
    free(s->Ru); free(s->Rv); free(s->fu); free(s->fv); free(s->us); free(s->vs);
    free(s->Ug); free(s->Vg); free(s->rhs); free(s->dp); free(s->cr); free(s->cz);
    free(s->cp); free(s->cq); free(s->diag); free(s->ub_next);
    free(s->nbE); free(s->nbW); free(s->nbN); free(s->nbS);
    free(s);
}

/* Load a state.  Unknown faces take the given values; inlet faces the inlet
 * profile; outlet faces the given value; wall / solid faces zero; periodic copy
 * faces mirror face 0.  p may be NULL (zero). Resets the step counter. */
void orc_set_state(orc_sim *s, const double *u, const double *v, const double *p)
{
    int nx = s->nx, ny = s->ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            size_t k = IU(s, i, j);
            switch (s->uk[k]) {
            case FK_UNKNOWN: case FK_OUTLET: s->u[k] = u[k]; break;
            case FK_INLET: s->u[k] = inlet_profile(s, j); break;
            default: s->u[k] = 0.0;
            }
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = IV(s, i, j);
            s->v[k] = (s->vk[k] == FK_UNKNOWN) ? v[k] : 0.0;
        }
    if (s->P.bc_x == 1) for (int j = 0; j < ny; ++j) s->u[IU(s, nx, j)] = s->u[IU(s, 0, j)];
    if (s->P.bc_y == 1) for (int i = 0; i < nx; ++i) s->v[IV(s, i, ny)] = s->v[IV(s, i, 0)];
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = IC(s, i, j);
            s->p[k] = (p && s->F[k]) ? p[k] : 0.0;
            s->dp[k] = 0.0;
        }
    memset(s->Ru, 0, sizeof(double) * (size_t)(nx + 1) * ny);
    memset(s->Rv, 0, sizeof(double) * (size_t)nx * (ny + 1));
    s->nstep = 0;
}

void orc_get_state(const orc_sim *s, double *u, double *v, double *p)
{
    size_t nc = (size_t)s->nx * s->ny, nu_ = (size_t)(s->nx + 1) * s->ny, nv_ = (size_t)s->nx * (s->ny + 1);
    if (u) memcpy(u, s->u, nu_ * sizeof(double));
    if (v) memcpy(v, s->v, nv_ * sizeof(double));
    if (p) memcpy(p, s->p, nc * sizeof(double));
}

void orc_set_face_forcing(orc_sim *s, const double *fu, const double *fv)
{
    size_t nu_ = (size_t)(s->nx + 1) * s->ny, nv_ = (size_t)s->nx * (s->ny + 1);
    for (size_t k = 0; k < nu_; ++k) s->fu[k] = (fu && s->uk[k] == FK_UNKNOWN) ? fu[k] : 0.0;
    for (size_t k = 0; k < nv_; ++k) s->fv[k] = (fv && s->vk[k] == FK_UNKNOWN) ? fv[k] : 0.0;
}

/* Reflection sign of the tangential velocity across a lower wall at face column i: -1 (no slip),
 * or +1 on the slip segments (Sec. 4.4). */
static double lower_wall_sign(const orc_sim *s, int i)
{
    if (!s->P.lip_slip) return -1.0;
    double x = s->P.x0 + (double)i * s->dx;
    return (x < s->P.slip_lo || x > s->P.slip_hi) ? 1.0 : -1.0;
}

/* --------------------------------------------------------------------- */
/* Ghost filling: copy the state into padded arrays, then give every      */
/* stencil position outside the fluid the value its boundary rule implies. */
/* --------------------------------------------------------------------- */
static void fill_ghosts(orc_sim *s, const double *u, const double *v)
{
    int nx = s->nx, ny = s->ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) UG(s, i, j) = u[IU(s, i, j)];
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) VG(s, i, j) = v[IV(s, i, j)];

    /* faces buried in solid: mirror of the fluid-side neighbour across the wall */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            if (s->uk[IU(s, i, j)] != FK_SOLID) continue;
            int up = (j + 1 < ny) && s->uk[IU(s, i, j + 1)] == FK_UNKNOWN;
            int dn = (j - 1 >= 0) && s->uk[IU(s, i, j - 1)] == FK_UNKNOWN;
            if (up && dn) { fprintf(stderr, "oracle: one-cell-thick solid layer is not supported\n"); abort(); }
            UG(s, i, j) = up ? lower_wall_sign(s, i) * u[IU(s, i, j + 1)] : (dn ? -u[IU(s, i, j - 1)] : 0.0);
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            if (s->vk[IV(s, i, j)] != FK_SOLID) continue;
            int rt = (i + 1 < nx) && s->vk[IV(s, i + 1, j)] == FK_UNKNOWN;
            int lt = (i - 1 >= 0) && s->vk[IV(s, i - 1, j)] == FK_UNKNOWN;
            if (rt && lt) { fprintf(stderr, "oracle: one-cell-thick solid layer is not supported\n"); abort(); }
            VG(s, i, j) = rt ? -v[IV(s, i + 1, j)] : (lt ? -v[IV(s, i - 1, j)] : 0.0);
        }

    /* x edges */
    for (int j = 0; j < ny; ++j) {
        if (s->P.bc_x == 1) {
            UG(s, nx, j) = UG(s, 0, j);
            UG(s, -1, j) = UG(s, nx - 1, j);
            UG(s, nx + 1, j) = UG(s, 1, j);
        } else {
            UG(s, -1, j) = 0.0;     /* never read: faces 0 and nx are boundary faces */
            UG(s, nx + 1, j) = 0.0;
        }
    }
    for (int j = 0; j <= ny; ++j) {
        if (s->P.bc_x == 1) {
            VG(s, -1, j) = VG(s, nx - 1, j);
            VG(s, nx, j) = VG(s, 0, j);
        } else {
            VG(s, -1, j) = -VG(s, 0, j);          /* inlet: v = 0 */
            VG(s, nx, j) = VG(s, nx - 1, j);      /* outlet: dv/dx = 0 */
        }
    }
    /* y edges (over the full padded width, so corners follow) */
    for (int i = -1; i <= nx + 1; ++i) {
        if (s->P.bc_y == 1) {
            UG(s, i, -1) = UG(s, i, ny - 1);
            UG(s, i, ny) = UG(s, i, 0);
        } else if (s->P.bc_y == 2) {
            UG(s, i, -1) = -UG(s, i, 0);
            UG(s, i, ny) = -UG(s, i, ny - 1);
        } else {
            UG(s, i, -1) = -UG(s, i, 0);          /* bottom: no slip */
            UG(s, i, ny) = UG(s, i, ny - 1);      /* top: free slip */
        }
    }
    for (int i = -1; i <= nx; ++i) {
        if (s->P.bc_y == 1) {
            VG(s, i, ny) = VG(s, i, 0);
            VG(s, i, -1) = VG(s, i, ny - 1);
            VG(s, i, ny + 1) = VG(s, i, 1);
        } else {
            VG(s, i, -1) = 0.0;                   /* never read */
            VG(s, i, ny + 1) = 0.0;
        }
    }
}

/* Explicit right-hand side of the momentum equations at the unknown faces:
 * R = -div(u u) + (1/Re) lap(u) + f   (central, divergence form). */
static void explicit_rhs(orc_sim *s, double *Ru_out, double *Rv_out)
{
    int nx = s->nx, ny = s->ny;
    double dx = s->dx, dy = s->dy, nu = s->nu;
    int adv = s->P.advection;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            size_t k = IU(s, i, j);
            if (s->uk[k] != FK_UNKNOWN) { Ru_out[k] = 0.0; continue; }
            double uc = UG(s, i, j), ue = UG(s, i + 1, j), uw = UG(s, i - 1, j);
            double un = UG(s, i, j + 1), us = UG(s, i, j - 1);
            double A = 0.0;
            if (adv) {
                double fe = 0.5 * (uc + ue), fw = 0.5 * (uw + uc);
                double un_c = 0.5 * (uc + un), vn_c = 0.5 * (VG(s, i - 1, j + 1) + VG(s, i, j + 1));
                double us_c = 0.5 * (us + uc), vs_c = 0.5 * (VG(s, i - 1, j) + VG(s, i, j));
                A = (fe * fe - fw * fw) / dx + (un_c * vn_c - us_c * vs_c) / dy;
            }
            double D = nu * ((ue - 2.0 * uc + uw) / (dx * dx) + (un - 2.0 * uc + us) / (dy * dy));
            Ru_out[k] = -A + D + s->fu[k];
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = IV(s, i, j);
            if (s->vk[k] != FK_UNKNOWN) { Rv_out[k] = 0.0; continue; }
            double vc = VG(s, i, j), ve = VG(s, i + 1, j), vw = VG(s, i - 1, j);
            double vn = VG(s, i, j + 1), vs = VG(s, i, j - 1);
            double A = 0.0;
            if (adv) {
                double ue_c = 0.5 * (UG(s, i + 1, j - 1) + UG(s, i + 1, j)), ve_c = 0.5 * (vc + ve);
                double uw_c = 0.5 * (UG(s, i, j - 1) + UG(s, i, j)), vw_c = 0.5 * (vw + vc);
                double fn = 0.5 * (vc + vn), fs = 0.5 * (vs + vc);
                A = (ue_c * ve_c - uw_c * vw_c) / dx + (fn * fn - fs * fs) / dy;
            }
            double D = nu * ((ve - 2.0 * vc + vw) / (dx * dx) + (vn - 2.0 * vc + vs) / (dy * dy));
            Rv_out[k] = -A + D + s->fv[k];
        }
}

/* ------------------------------ Poisson ------------------------------- */
/* Connectivity of fluid cell (i,j) to its east / north neighbour: the face
 * between them is an unknown. */
static int conn_e(const orc_sim *s, int i, int j)
{
    int f = i + 1;
    if (s->P.bc_x == 1) f = wrap(f, s->nx); else if (f >= s->nx) return 0;
    return s->uk[IU(s, f, j)] == FK_UNKNOWN;
}
static int conn_w(const orc_sim *s, int i, int j)
{
    if (s->P.bc_x != 1 && i == 0) return 0;
    return s->uk[IU(s, (s->P.bc_x == 1) ? wrap(i, s->nx) : i, j)] == FK_UNKNOWN;
}
static int conn_n(const orc_sim *s, int i, int j)
{
    int f = j + 1;
    if (s->P.bc_y == 1) f = wrap(f, s->ny); else if (f >= s->ny) return 0;
    return s->vk[IV(s, i, f)] == FK_UNKNOWN;
}
static int conn_s(const orc_sim *s, int i, int j)
{
    if (s->P.bc_y != 1 && j == 0) return 0;
    return s->vk[IV(s, i, (s->P.bc_y == 1) ? wrap(j, s->ny) : j)] == FK_UNKNOWN;
}

/* y = (-L) x on fluid cells: sum over connected neighbours of (x_c - x_nb)/h^2 */
static void apply_negL(const orc_sim *s, const double *x, double *y)
{
    size_t nc = (size_t)s->nx * s->ny;
    double ax = 1.0 / (s->dx * s->dx), ay = 1.0 / (s->dy * s->dy);
    for (size_t k = 0; k < nc; ++k) {
        if (!s->F[k]) { y[k] = 0.0; continue; }
        double xc = x[k], acc = 0.0;
        if (s->nbE[k] >= 0) acc += ax * (xc - x[s->nbE[k]]);
        if (s->nbW[k] >= 0) acc += ax * (xc - x[s->nbW[k]]);
        if (s->nbN[k] >= 0) acc += ay * (xc - x[s->nbN[k]]);
        if (s->nbS[k] >= 0) acc += ay * (xc - x[s->nbS[k]]);
        y[k] = acc;
    }
}

static void make_diag(orc_sim *s)
{
    size_t nc = (size_t)s->nx * s->ny;
    double ax = 1.0 / (s->dx * s->dx), ay = 1.0 / (s->dy * s->dy);
    for (size_t k = 0; k < nc; ++k) {
        double d = 0.0;
        if (s->F[k]) {
            d += (s->nbE[k] >= 0) ? ax : 0.0;
            d += (s->nbW[k] >= 0) ? ax : 0.0;
            d += (s->nbN[k] >= 0) ? ay : 0.0;
            d += (s->nbS[k] >= 0) ? ay : 0.0;
        }
        s->diag[k] = d;
    }
}

static double dot_fluid(const orc_sim *s, const double *a, const double *b)
{
    double acc = 0.0;
    size_t nc = (size_t)s->nx * s->ny;
    for (size_t k = 0; k < nc; ++k) if (s->F[k]) acc += a[k] * b[k];
    return acc;
}

static void remove_mean(const orc_sim *s, double *x)
{
    size_t nc = (size_t)s->nx * s->ny;
    double sum = 0.0; long n = 0;
    for (size_t k = 0; k < nc; ++k) if (s->F[k]) { sum += x[k]; ++n; }
    if (n == 0) return;
    double m = sum / (double)n;
    for (size_t k = 0; k < nc; ++k) x[k] = s->F[k] ? x[k] - m : 0.0;
}

/* Solve (-L) x = rhs with Jacobi-preconditioned CG, x as initial guess.
 * rhs must be mean-zero on fluid cells.  Returns iterations. */
static int pcg_solve(orc_sim *s, const double *rhs, double *x)
{
    size_t nc = (size_t)s->nx * s->ny;
    double *r = s->cr, *z = s->cz, *p = s->cp, *q = s->cq;
    make_diag(s);
    double bnorm = sqrt(dot_fluid(s, rhs, rhs));
    if (bnorm == 0.0) {
        for (size_t k = 0; k < nc; ++k) x[k] = 0.0;
        s->last_cg_relres = 0.0;
        return 0;
    }
    apply_negL(s, x, q);
    for (size_t k = 0; k < nc; ++k) r[k] = s->F[k] ? rhs[k] - q[k] : 0.0;
    for (size_t k = 0; k < nc; ++k) z[k] = (s->diag[k] > 0.0) ? r[k] / s->diag[k] : 0.0;
    memcpy(p, z, nc * sizeof(double));
    double rz = dot_fluid(s, r, z);
    int it = 0;
    double rn = sqrt(dot_fluid(s, r, r));
    while (rn > s->P.cg_rtol * bnorm && it < s->P.cg_maxit) {
        apply_negL(s, p, q);
        double pq = dot_fluid(s, p, q);
        if (pq <= 0.0) break;
        double alpha = rz / pq;
        for (size_t k = 0; k < nc; ++k) { x[k] += alpha * p[k]; r[k] -= alpha * q[k]; }
        ++it;
        rn = sqrt(dot_fluid(s, r, r));
        if (rn <= s->P.cg_rtol * bnorm) break;
        for (size_t k = 0; k < nc; ++k) z[k] = (s->diag[k] > 0.0) ? r[k] / s->diag[k] : 0.0;
        double rz1 = dot_fluid(s, r, z);
        double beta = rz1 / rz;
        rz = rz1;
        for (size_t k = 0; k < nc; ++k) p[k] = z[k] + beta * p[k];
    }
    s->last_cg_relres = rn / bnorm;
    return it;
}

/* rhs = (D u)/dt on fluid cells */
static void divergence(const orc_sim *s, const double *u, const double *v, double scale, double *out)
{
    int nx = s->nx, ny = s->ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = IC(s, i, j);
            if (!s->F[k]) { out[k] = 0.0; continue; }
            double d = (u[IU(s, i + 1, j)] - u[IU(s, i, j)]) / s->dx + (v[IV(s, i, j + 1)] - v[IV(s, i, j)]) / s->dy;
            out[k] = scale * d;
        }
}

/* Gradient correction u -= c * G phi at unknown faces (periodic copies kept). */
static void grad_correct(orc_sim *s, double *u, double *v, const double *phi, double c)
{
    int nx = s->nx, ny = s->ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            size_t k = IU(s, i, j);
            if (s->uk[k] != FK_UNKNOWN) continue;
            double g = (phi[IC(s, wrap(i, nx), j)] - phi[IC(s, wrap(i - 1, nx), j)]) / s->dx;
            u[k] -= c * g;
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = IV(s, i, j);
            if (s->vk[k] != FK_UNKNOWN) continue;
            double g = (phi[IC(s, i, wrap(j, ny))] - phi[IC(s, i, wrap(j - 1, ny))]) / s->dy;
            v[k] -= c * g;
        }
    if (s->P.bc_x == 1) for (int j = 0; j < ny; ++j) u[IU(s, nx, j)] = u[IU(s, 0, j)];
    if (s->P.bc_y == 1) for (int i = 0; i < nx; ++i) v[IV(s, i, ny)] = v[IV(s, i, 0)];
}

/* Convective outflow (left / right boundaries of bc_x == 0). */
static void outlet_update(orc_sim *s)
{
    if (s->P.bc_x != 0) return;
    int nx = s->nx, ny = s->ny;
    double qin = 0.0, qout = 0.0;
    int nout = 0;
    for (int j = 0; j < ny; ++j) {
        if (s->uk[IU(s, 0, j)] == FK_INLET) qin += inlet_profile(s, j) * s->dy;
        if (s->uk[IU(s, nx, j)] == FK_OUTLET) {
            double ub = s->u[IU(s, nx, j)], ui = s->u[IU(s, nx - 1, j)];
            s->ub_next[j] = ub - s->P.dt * s->P.conv_speed * (ub - ui) / s->dx;
            qout += s->ub_next[j] * s->dy;
            ++nout;
        } else {
            s->ub_next[j] = 0.0;
        }
    }
    if (nout > 0) {
        double shift = (qin - qout) / ((double)nout * s->dy);
        for (int j = 0; j < ny; ++j)
            if (s->uk[IU(s, nx, j)] == FK_OUTLET) s->ub_next[j] += shift;
    }
}

/* One time step n -> n+1. */
static void step_once(orc_sim *s)
{
    int nx = s->nx, ny = s->ny;
    double dt = s->P.dt;
    size_t nu_ = (size_t)(nx + 1) * ny, nv_ = (size_t)nx * (ny + 1);
    double c1 = (s->nstep == 0) ? 1.0 : 1.5, c0 = (s->nstep == 0) ? 0.0 : -0.5;

    outlet_update(s);
    fill_ghosts(s, s->u, s->v);
    /* R^n into us/vs temporarily */
    explicit_rhs(s, s->us, s->vs);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            size_t k = IU(s, i, j);
            double Rn = s->us[k];
            switch (s->uk[k]) {
            case FK_UNKNOWN: {
                double gp = (s->p[IC(s, wrap(i, nx), j)] - s->p[IC(s, wrap(i - 1, nx), j)]) / s->dx;
                s->us[k] = s->u[k] + dt * (c1 * Rn + c0 * s->Ru[k]) - dt * gp;
                s->Ru[k] = Rn;
                break;
            }
            case FK_INLET: s->us[k] = inlet_profile(s, j); break;
            case FK_OUTLET: s->us[k] = s->ub_next[j]; break;
            default: s->us[k] = 0.0;
            }
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = IV(s, i, j);
            double Rn = s->vs[k];
            if (s->vk[k] == FK_UNKNOWN) {
                double gp = (s->p[IC(s, i, wrap(j, ny))] - s->p[IC(s, i, wrap(j - 1, ny))]) / s->dy;
                s->vs[k] = s->v[k] + dt * (c1 * Rn + c0 * s->Rv[k]) - dt * gp;
                s->Rv[k] = Rn;
            } else {
                s->vs[k] = 0.0;
            }
        }
    if (s->P.bc_x == 1) for (int j = 0; j < ny; ++j) s->us[IU(s, nx, j)] = s->us[IU(s, 0, j)];
    if (s->P.bc_y == 1) for (int i = 0; i < nx; ++i) s->vs[IV(s, i, ny)] = s->vs[IV(s, i, 0)];

    /* pressure increment: L dp = D u* / dt  <=>  (-L) dp = -D u* / dt */
    divergence(s, s->us, s->vs, -1.0 / dt, s->rhs);
    remove_mean(s, s->rhs);
    s->last_cg_iters = pcg_solve(s, s->rhs, s->dp);
    remove_mean(s, s->dp);

    grad_correct(s, s->us, s->vs, s->dp, dt);
    memcpy(s->u, s->us, nu_ * sizeof(double));
    memcpy(s->v, s->vs, nv_ * sizeof(double));
    size_t nc = (size_t)nx * ny;
    for (size_t k = 0; k < nc; ++k) if (s->F[k]) s->p[k] += s->dp[k];
    s->nstep += 1;
}

int orc_step(orc_sim *s, int nsteps)
{
    int total = 0;
    for (int n = 0; n < nsteps; ++n) { step_once(s); total += s->last_cg_iters; }
    return total;
}

double orc_max_div(const orc_sim *s)
{
    double m = 0.0;
    for (int j = 0; j < s->ny; ++j)
        for (int i = 0; i < s->nx; ++i) {
            if (!s->F[IC(s, i, j)]) continue;
            double d = (s->u[IU(s, i + 1, j)] - s->u[IU(s, i, j)]) / s->dx + (s->v[IV(s, i, j + 1)] - s->v[IV(s, i, j)]) / s->dy;
            if (fabs(d) > m) m = fabs(d);
        }
    return m;
}

double orc_last_cg_relres(const orc_sim *s) { return s->last_cg_relres; }
int orc_last_cg_iters(const orc_sim *s) { return s->last_cg_iters; }

/* Inflow and outflow volume fluxes (per unit depth) of the current state. */
void orc_fluxes(const orc_sim *s, double *qin, double *qout)
{
    double a = 0.0, b = 0.0;
    for (int j = 0; j < s->ny; ++j) {
        a += s->u[IU(s, 0, j)] * s->dy;
        b += s->u[IU(s, s->nx, j)] * s->dy;
    }
    *qin = a; *qout = b;
}

/* Face kinds, for tests: u kinds (nx+1)*ny then v kinds nx*(ny+1). */
void orc_face_kinds(const orc_sim *s, unsigned char *uk, unsigned char *vk)
{
    memcpy(uk, s->uk, (size_t)(s->nx + 1) * s->ny);
    memcpy(vk, s->vk, (size_t)s->nx * (s->ny + 1));
}

/* Apply the discrete projection P = I - G (DG)^{-1} D to a face field (no time
 * step, no boundary update); boundary faces are left unchanged. */
void orc_project(orc_sim *s, double *u, double *v)
{
    size_t nc = (size_t)s->nx * s->ny;
    divergence(s, u, v, -1.0, s->rhs);
    remove_mean(s, s->rhs);
    for (size_t k = 0; k < nc; ++k) s->dp[k] = 0.0;
    s->last_cg_iters = pcg_solve(s, s->rhs, s->dp);
    remove_mean(s, s->dp);
    grad_correct(s, u, v, s->dp, 1.0);
}

/* Poisson pieces exposed for tests: y = (-L) x, and x = (-L)^+ b (mean-zero). */
void orc_apply_negL(orc_sim *s, const double *x, double *y) { apply_negL(s, x, y); }
int orc_poisson_solve(orc_sim *s, const double *b, double *x)
{
    size_t nc = (size_t)s->nx * s->ny;
    memcpy(s->rhs, b, nc * sizeof(double));
    remove_mean(s, s->rhs);
    for (size_t k = 0; k < nc; ++k) x[k] = 0.0;
    int it = pcg_solve(s, s->rhs, x);
    remove_mean(s, x);
    return it;
}
/* Explicit right-hand side R(u) + f of the current state (tests). */
void orc_explicit_rhs(orc_sim *s, double *Ru, double *Rv)
{
    fill_ghosts(s, s->u, s->v);
    explicit_rhs(s, Ru, Rv);
}

/* ------------------------- control and ensemble ------------------------ */
/* Control region (Sec. 4.1): cells whose centre lies in [rx0,rx1] x [ry0,ry1]
 * (inclusive).  Fills rect = {ia, ib, ja, jb}; returns 0, or -1 if empty. */
int orc_control_rect(const orc_params *P, const double *region, int *rect)
{
    int ia = -1, ib = -1, ja = -1, jb = -1;
    for (int i = 0; i < P->nx; ++i) {
        double xc = orc_cell_xc(P, i);
        if (xc >= region[0] && xc <= region[1]) { if (ia < 0) ia = i; ib = i; }
    }
    for (int j = 0; j < P->ny; ++j) {
        double yc = orc_cell_yc(P, j);
        if (yc >= region[2] && yc <= region[3]) { if (ja < 0) ja = j; jb = j; }
    }
    rect[0] = ia; rect[1] = ib; rect[2] = ja; rect[3] = jb;
    return (ia < 0 || ja < 0) ? -1 : 0;
}

/* Control cells = fluid cells of the rectangle, row-major (j outer, i inner).
 * Returns their count; fills ci/cj if non-NULL. */
int orc_control_cells(const orc_params *P, const double *region, int *ci, int *cj)
{
    int rect[4];
    if (orc_control_rect(P, region, rect) != 0) return 0;
    unsigned char *F = (unsigned char *)xcalloc((size_t)P->nx * P->ny, 1);
    orc_fluid_mask(P, F);
    int n = 0;
    for (int j = rect[2]; j <= rect[3]; ++j)
        for (int i = rect[0]; i <= rect[1]; ++i)
            if (F[(size_t)j * P->nx + i]) {
                if (ci) ci[n] = i;
                if (cj) cj[n] = j;
                ++n;
            }
    free(F);
    return n;
}

/* The operator P of Eq. (discrete_NS): control vector f = [fx(cells), fy(cells)]
 * (cell-centred) -> face forcing by averaging the two cells adjacent to each
 * unknown face (cells outside the control set contribute zero). */
void orc_control_to_faces(const orc_params *P, const double *region, const double *f, double *fu, double *fv)
{
    int nx = P->nx, ny = P->ny;
    int nc = orc_control_cells(P, region, NULL, NULL);
    int *ci = (int *)xcalloc((size_t)nc, sizeof(int)), *cj = (int *)xcalloc((size_t)nc, sizeof(int));
    orc_control_cells(P, region, ci, cj);
    double *FX = (double *)xcalloc((size_t)nx * ny, sizeof(double));
    double *FY = (double *)xcalloc((size_t)nx * ny, sizeof(double));
    for (int c = 0; c < nc; ++c) {
        FX[(size_t)cj[c] * nx + ci[c]] = f[c];
        FY[(size_t)cj[c] * nx + ci[c]] = f[nc + c];
    }
    orc_sim *s = orc_create(P);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            size_t k = (size_t)j * (nx + 1) + i;
            fu[k] = 0.0;
            if (s->uk[k] != FK_UNKNOWN) continue;
            int il = wrap(i - 1, nx), ir = wrap(i, nx);
            fu[k] = 0.5 * (FX[(size_t)j * nx + il] + FX[(size_t)j * nx + ir]);
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = (size_t)j * nx + i;
            fv[k] = 0.0;
            if (s->vk[k] != FK_UNKNOWN) continue;
            int jl = wrap(j - 1, ny), jr = wrap(j, ny);
            fv[k] = 0.5 * (FY[(size_t)jl * nx + i] + FY[(size_t)jr * nx + i]);
        }
    orc_destroy(s);
    free(FX); free(FY); free(ci); free(cj);
}

/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
 * 4x64 Philox S-P network with the published multipliers and Weyl key
 * increments. */
void orc_philox4x64_10(const uint64_t *ctr_in, const uint64_t *key_in, uint64_t *out)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        unsigned __int128 p0 = (unsigned __int128)M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Standard normals number q = first .. first+n-1 of stream (seed, stream):
 * block b = q/4 is Philox4x64-10 of counter (b,0,0,0), key (seed, stream);
 * words (w0,w1) and (w2,w3) give two Box-Muller pairs:
 *   u1 = (w>>11 + 1) 2^-53 in (0,1],  u2 = (w>>11) 2^-53 in [0,1),
 *   z = sqrt(-2 ln u1) * (cos 2 pi u2, sin 2 pi u2). */
void orc_normals(uint64_t seed, uint64_t stream, int64_t first, int64_t n, double *out)
{
    const double two_m53 = 1.0 / 9007199254740992.0;
    const double twopi = 6.283185307179586476925286766559;
    for (int64_t t = 0; t < n; ++t) {
        int64_t q = first + t;
        uint64_t ctr[4] = {(uint64_t)(q / 4), 0, 0, 0}, key[2] = {seed, stream}, w[4];
        orc_philox4x64_10(ctr, key, w);
        int lane = (int)(q % 4);
        uint64_t a = (lane < 2) ? w[0] : w[2], b = (lane < 2) ? w[1] : w[3];
        double u1 = ((double)(a >> 11) + 1.0) * two_m53;
        double u2 = (double)(b >> 11) * two_m53;
        double rad = sqrt(-2.0 * log(u1));
        out[t] = (lane % 2 == 0) ? rad * cos(twopi * u2) : rad * sin(twopi * u2);
    }
}

/* White-noise convolution sampler for N(0, B), B_ij = sigma^2 exp(-dx^2/a^2 - dy^2/a^2)
 * (Eq. covarianceB with a_x = a_y = a, c_xy = infinity).
 * Along each axis, a lattice xi_k of spacing eta = h/m (m = ceil(4h/a), so eta <= a/4)
 * that contains the rectangle's cell centres and extends 5a beyond them carries
 * white noise; G[r][k] = c exp(-2 (x_r - xi_k)^2 / a^2), c^2 = 2 eta /(a sqrt(pi)).
 * Then sum_k G[r][k] G[s][k] = exp(-(x_r - x_s)^2 / a^2) up to the lattice
 * quadrature error (below 1e-16 for eta <= a/4) and the tail (exp(-50)).
 * orc_sampler_dims gives {nrx, nry, nxix, nxiy}. */
static void sampler_axis(double h, double a, int ncell, int *m_out, int *pad_out, int *nxi_out)
{
    int m = (int)ceil(4.0 * h / a);
    if (m < 1) m = 1;
    double eta = h / m;
    int pad = (int)ceil(5.0 * a / eta);
    *m_out = m; *pad_out = pad; *nxi_out = (ncell - 1) * m + 1 + 2 * pad;
}

int orc_sampler_dims(const orc_params *P, const double *region, double a, int *dims)
{
    int rect[4];
    if (orc_control_rect(P, region, rect) != 0) return -1;
    double dx = (P->x1 - P->x0) / P->nx, dy = (P->y1 - P->y0) / P->ny;
    int mx, px, nxix, my, py, nxiy;
    sampler_axis(dx, a, rect[1] - rect[0] + 1, &mx, &px, &nxix);
    sampler_axis(dy, a, rect[3] - rect[2] + 1, &my, &py, &nxiy);
    dims[0] = rect[1] - rect[0] + 1; dims[1] = rect[3] - rect[2] + 1;
    dims[2] = nxix; dims[3] = nxiy;
    return 0;
}

static void axis_factor(double h, double a, double first_centre, int ncell, double *G)
{
    int m, pad, nxi;
    sampler_axis(h, a, ncell, &m, &pad, &nxi);
    double eta = h / m;
    double c = sqrt(2.0 * eta / (a * sqrt(M_PI)));
    for (int r = 0; r < ncell; ++r) {
        double xr = first_centre + r * h;
        for (int k = 0; k < nxi; ++k) {
            double xi = first_centre + (double)(k - pad) * eta;
            double d = xr - xi;
            G[(size_t)r * nxi + k] = c * exp(-2.0 * d * d / (a * a));
        }
    }
}

/* The two 1-D factors (row-major [ncell][nxi]). */
int orc_sampler_factors(const orc_params *P, const double *region, double a, double *Gx, double *Gy)
{
    int rect[4], dims[4];
    if (orc_sampler_dims(P, region, a, dims) != 0) return -1;
    orc_control_rect(P, region, rect);
    double dx = (P->x1 - P->x0) / P->nx, dy = (P->y1 - P->y0) / P->ny;
    axis_factor(dx, a, orc_cell_xc(P, rect[0]), dims[0], Gx);
    axis_factor(dy, a, orc_cell_yc(P, rect[2]), dims[1], Gy);
    return 0;
}

/* Ensemble from given white noise Z, layout [member][component][nxiy][nxix].
 * E is n_ctrl x N column-major (n_ctrl = 2 * control cells; fx block first):
 * E[(c, cell), k] = sigma * sum_{kx,ky} Gx[ix][kx] Gy[iy][ky] Z[k][c][ky][kx]. */
int orc_ensemble_from_noise(const orc_params *P, const double *region, double sigma, double a, int N,
                            const double *Z, double *E)
{
    int dims[4], rect[4];
    if (orc_sampler_dims(P, region, a, dims) != 0) return -1;
    orc_control_rect(P, region, rect);
    int nrx = dims[0], nry = dims[1], nxix = dims[2], nxiy = dims[3];
    int ncc = orc_control_cells(P, region, NULL, NULL);
    int *ci = (int *)xcalloc((size_t)ncc, sizeof(int)), *cj = (int *)xcalloc((size_t)ncc, sizeof(int));
    orc_control_cells(P, region, ci, cj);
    double *Gx = (double *)xcalloc((size_t)nrx * nxix, sizeof(double));
    double *Gy = (double *)xcalloc((size_t)nry * nxiy, sizeof(double));
    orc_sampler_factors(P, region, a, Gx, Gy);
    double *T = (double *)xcalloc((size_t)nxiy * nrx, sizeof(double));   /* T[ky][ix] */
    size_t nctrl = 2 * (size_t)ncc;
    for (int k = 0; k < N; ++k)
        for (int c = 0; c < 2; ++c) {
            const double *Zk = Z + ((size_t)k * 2 + c) * (size_t)nxiy * nxix;
            /* contract x first */
            for (int ky = 0; ky < nxiy; ++ky)
                for (int ix = 0; ix < nrx; ++ix) {
                    double acc = 0.0;
                    for (int kx = 0; kx < nxix; ++kx) acc += Gx[(size_t)ix * nxix + kx] * Zk[(size_t)ky * nxix + kx];
                    T[(size_t)ky * nrx + ix] = acc;
                }
            for (int q = 0; q < ncc; ++q) {
                int ix = ci[q] - rect[0], iy = cj[q] - rect[2];
                double acc = 0.0;
                for (int ky = 0; ky < nxiy; ++ky) acc += Gy[(size_t)iy * nxiy + ky] * T[(size_t)ky * nrx + ix];
                E[(size_t)k * nctrl + (size_t)c * ncc + q] = sigma * acc;
            }
        }
    free(T); free(Gx); free(Gy); free(ci); free(cj);
    return 0;
}

/* Seeded ensemble: Z drawn with orc_normals(seed, stream = 0), normal index =
 * position in the [member][component][nxiy][nxix] layout. */
int orc_ensemble_seeded(const orc_params *P, const double *region, double sigma, double a, int N,
                        uint64_t seed, double *E)
{
    int dims[4];
    if (orc_sampler_dims(P, region, a, dims) != 0) return -1;
    int64_t nz = (int64_t)N * 2 * dims[2] * dims[3];
    double *Z = (double *)xcalloc((size_t)nz, sizeof(double));
    orc_normals(seed, 0, 0, nz, Z);
    int rc = orc_ensemble_from_noise(P, region, sigma, a, N, Z, E);
    free(Z);
    return rc;
}

/* ------------------------------- costs --------------------------------- */
static double interp_u(const orc_sim *s, double x, double y)
{
    double fi = (x - s->P.x0) / s->dx, fj = (y - s->P.y0) / s->dy - 0.5;
    int i0 = (int)floor(fi), j0 = (int)floor(fj);
    if (i0 < 0 || i0 + 1 > s->nx || j0 < 0 || j0 + 1 > s->ny - 1) return NAN;
    double tx = fi - i0, ty = fj - j0;
    const double *u = s->u;
    return (1 - tx) * (1 - ty) * u[IU(s, i0, j0)] + tx * (1 - ty) * u[IU(s, i0 + 1, j0)]
         + (1 - tx) * ty * u[IU(s, i0, j0 + 1)] + tx * ty * u[IU(s, i0 + 1, j0 + 1)];
}
static double interp_v(const orc_sim *s, double x, double y)
{
    double fi = (x - s->P.x0) / s->dx - 0.5, fj = (y - s->P.y0) / s->dy;
    int i0 = (int)floor(fi), j0 = (int)floor(fj);
    if (i0 < 0 || i0 + 1 > s->nx - 1 || j0 < 0 || j0 + 1 > s->ny) return NAN;
    double tx = fi - i0, ty = fj - j0;
    const double *v = s->v;
    double a = (1 - tx) * v[IV(s, i0, j0)] + tx * v[IV(s, i0 + 1, j0)];
    double b = (ty > 0.0) ? (1 - tx) * v[IV(s, i0, j0 + 1)] + tx * v[IV(s, i0 + 1, j0 + 1)] : 0.0;
    return (1 - ty) * a + ty * b;
}

/* Sensors of Sec. 4.1: x = 1/5, 2/5, 3/5, 4/5 at y = 0; out[2s] = u, out[2s+1] = v. */
void orc_sensors(const orc_sim *s, double *out)
{
    for (int q = 0; q < 4; ++q) {
        double x = 0.2 * (q + 1);
        out[2 * q] = interp_u(s, x, 0.0);
        out[2 * q + 1] = interp_v(s, x, 0.0);
    }
}

typedef struct {
    double *u, *v, *p, *Ru, *Rv, *dp;
    long nstep;
} snapshot;

static void snap_take(const orc_sim *s, snapshot *q)
{
    size_t nc = (size_t)s->nx * s->ny, nu_ = (size_t)(s->nx + 1) * s->ny, nv_ = (size_t)s->nx * (s->ny + 1);
    q->u = (double *)xcalloc(nu_, sizeof(double)); memcpy(q->u, s->u, nu_ * sizeof(double));
    q->v = (double *)xcalloc(nv_, sizeof(double)); memcpy(q->v, s->v, nv_ * sizeof(double));
    q->Ru = (double *)xcalloc(nu_, sizeof(double)); memcpy(q->Ru, s->Ru, nu_ * sizeof(double));
    q->Rv = (double *)xcalloc(nv_, sizeof(double)); memcpy(q->Rv, s->Rv, nv_ * sizeof(double));
    q->p = (double *)xcalloc(nc, sizeof(double)); memcpy(q->p, s->p, nc * sizeof(double));
    q->dp = (double *)xcalloc(nc, sizeof(double)); memcpy(q->dp, s->dp, nc * sizeof(double));
    q->nstep = s->nstep;
}
static void snap_restore(orc_sim *s, const snapshot *q)
{
    size_t nc = (size_t)s->nx * s->ny, nu_ = (size_t)(s->nx + 1) * s->ny, nv_ = (size_t)s->nx * (s->ny + 1);
    memcpy(s->u, q->u, nu_ * sizeof(double)); memcpy(s->v, q->v, nv_ * sizeof(double));
    memcpy(s->Ru, q->Ru, nu_ * sizeof(double)); memcpy(s->Rv, q->Rv, nv_ * sizeof(double));
    memcpy(s->p, q->p, nc * sizeof(double)); memcpy(s->dp, q->dp, nc * sizeof(double));
    s->nstep = q->nstep;
}
static void snap_free(snapshot *q) { free(q->u); free(q->v); free(q->p); free(q->Ru); free(q->Rv); free(q->dp); }

/* Run one member from the raw initial fields (u0, v0) with face forcing (fu, fv)
 * over n_steps, the last n_window of which form the cost window.  Costs by the
 * two-pass definition (window means first, then squared deviations; the window
 * is re-run from a snapshot so that the trajectory is identical):
 *   J_domain = (1/(2 n_w)) sum_cells dx dy sum_t |u_c(t) - mean u_c|^2,
 *   J_sensor = 1/2 sum_sensors sum_t |u(x_s, t) - mean u(x_s)|^2.
 * series (may be NULL) receives the sensor samples [n_window][8].
 * u_end/v_end/p_end (may be NULL) receive the final state.  Returns 0. */
int orc_member_run(const orc_params *P, const double *u0, const double *v0, const double *fu, const double *fv,
                   int n_steps, int n_window, double *J_domain, double *J_sensor, double *series,
                   double *u_end, double *v_end, double *p_end, double *max_div)
{
    if (n_window > n_steps || n_window < 0) return -1;
    orc_sim *s = orc_create(P);
    if (!s) return -2;
    orc_set_state(s, u0, v0, NULL);
    orc_set_face_forcing(s, fu, fv);
    int nx = s->nx, ny = s->ny;
    size_t nc = (size_t)nx * ny;
    double md = 0.0;
    int nw0 = n_steps - n_window;
    orc_step(s, nw0);
    if (nw0 > 0 && orc_max_div(s) > md) md = orc_max_div(s);
    snapshot snap;
    snap_take(s, &snap);
    double *mu = (double *)xcalloc(nc, sizeof(double)), *mv = (double *)xcalloc(nc, sizeof(double));
    double *ser = (double *)xcalloc((size_t)(n_window > 0 ? n_window : 1) * 8, sizeof(double));
    for (int t = 0; t < n_window; ++t) {
        step_once(s);
        double d = orc_max_div(s); if (d > md) md = d;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t k = IC(s, i, j);
                if (!s->F[k]) continue;
                mu[k] += 0.5 * (s->u[IU(s, i, j)] + s->u[IU(s, i + 1, j)]);
                mv[k] += 0.5 * (s->v[IV(s, i, j)] + s->v[IV(s, i, j + 1)]);
            }
        orc_sensors(s, ser + (size_t)t * 8);
    }
    if (u_end || v_end || p_end) orc_get_state(s, u_end, v_end, p_end);
    double jd = 0.0;
    if (n_window > 0) {
        for (size_t k = 0; k < nc; ++k) { mu[k] /= n_window; mv[k] /= n_window; }
        snap_restore(s, &snap);
        double *acc = (double *)xcalloc(nc, sizeof(double));
        for (int t = 0; t < n_window; ++t) {
            step_once(s);
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t k = IC(s, i, j);
                    if (!s->F[k]) continue;
                    double a = 0.5 * (s->u[IU(s, i, j)] + s->u[IU(s, i + 1, j)]) - mu[k];
                    double b = 0.5 * (s->v[IV(s, i, j)] + s->v[IV(s, i, j + 1)]) - mv[k];
                    acc[k] += a * a + b * b;
                }
        }
        for (size_t k = 0; k < nc; ++k) jd += acc[k];
        jd *= s->dx * s->dy / (2.0 * n_window);
        free(acc);
    }
    double js = 0.0;
    if (n_window > 0) {
        for (int c = 0; c < 8; ++c) {
            double m = 0.0;
            for (int t = 0; t < n_window; ++t) m += ser[(size_t)t * 8 + c];
            m /= n_window;
            for (int t = 0; t < n_window; ++t) { double d = ser[(size_t)t * 8 + c] - m; js += d * d; }
        }
        js *= 0.5;
    }
    if (series) memcpy(series, ser, (size_t)n_window * 8 * sizeof(double));
    if (J_domain) *J_domain = jd;
    if (J_sensor) *J_sensor = js;
    if (max_div) *max_div = md;
    free(mu); free(mv); free(ser);
    snap_free(&snap);
    orc_destroy(s);
    return 0;
}

/* Trajectory only: n_steps from the raw initial fields, final state out. */
int orc_trajectory(const orc_params *P, const double *u0, const double *v0, const double *p0,
                   const double *fu, const double *fv, int n_steps,
                   double *u_end, double *v_end, double *p_end, double *max_div, int *cg_iters)
{
    orc_sim *s = orc_create(P);
    if (!s) return -2;
    orc_set_state(s, u0, v0, p0);
    orc_set_face_forcing(s, fu, fv);
    double md = 0.0;
    int it = 0;
    for (int n = 0; n < n_steps; ++n) {
        step_once(s);
        it += s->last_cg_iters;
        double d = orc_max_div(s); if (d > md) md = d;
    }
    orc_get_state(s, u_end, v_end, p_end);
    if (max_div) *max_div = md;
    if (cg_iters) *cg_iters = it;
    orc_destroy(s);
    return 0;
}

/* ------------------------------- EnVar --------------------------------- */
/* Eq. (gradient_EnVar) with the columns of Y from Eq. (fdapprox), contracted
 * with R^{-1}(Hq - y) through the scalar cost: for J_obs = 1/2 ||Hq - y||^2,
 * (J_obs(f + eps E_i) - J_obs(f)) / eps = Y_i^T (Hq - y) + O(eps), so
 *   g_i = (J_i - J_0)/eps + (N - 1) w_i.  Also returns J_prior = (N-1)/2 w^T w. */
void orc_gradient_from_costs(int N, const double *J, const double *w, double eps, double *g, double *J_prior)
{
    double jp = 0.0;
    for (int i = 0; i < N; ++i) {
        g[i] = (J[i + 1] - J[0]) / eps + (double)(N - 1) * w[i];
        jp += w[i] * w[i];
    }
    if (J_prior) *J_prior = 0.5 * (double)(N - 1) * jp;
}

/* Eq. (gradient_EnVar) with Y built column by column from Eq. (fdapprox) on the
 * sensor observations of Sec. 4.1 (R = I, y = 0): H q_m = u'_m(x_s, t_j), the
 * fluctuation about the member's own window mean, for s = 1..4 sensors x 2
 * components and every window step;  Y_i = (H q_i - H q_0)/eps,
 * g = Y^T (H q_0 - y) + (N-1) w.   series: [N+1][n_window][8]. */
void orc_sensor_gradient(int N, int n_window, const double *series, double eps, const double *w, double *g)
{
    size_t nobs = (size_t)n_window * 8;
    double *h0 = (double *)xcalloc(nobs, sizeof(double)), *hi = (double *)xcalloc(nobs, sizeof(double));
    for (int m = 0; m <= N; ++m) {
        double *h = (m == 0) ? h0 : hi;
        const double *sm = series + (size_t)m * nobs;
        for (int c = 0; c < 8; ++c) {
            double mean = 0.0;
            for (int t = 0; t < n_window; ++t) mean += sm[(size_t)t * 8 + c];
            mean /= n_window;
            for (int t = 0; t < n_window; ++t) h[(size_t)t * 8 + c] = sm[(size_t)t * 8 + c] - mean;
        }
        if (m == 0) continue;
        double acc = 0.0;
        for (size_t k = 0; k < nobs; ++k) acc += (hi[k] - h0[k]) / eps * h0[k];
        g[m - 1] = acc + (double)(N - 1) * w[m - 1];
    }
    free(h0); free(hi);
}

/* Weight update of Sec. 3.3.1 with the step preconditioned by the prior Hessian (N-1) I of
 * Eq. (J_w):  w <- w - alpha g / (N-1).  Also the total cost of Eq. (J_w) at the old w,
 * J(w) = J_obs(member 0) + (N-1)/2 w^T w.  w_out may alias w. */
void orc_envar_step(int N, const double *w, const double *g, double alpha, double J0_obs, double *w_out,
                    double *J_total)
{
    double ww = 0.0;
    for (int i = 0; i < N; ++i) ww += w[i] * w[i];
    double denom = (N > 1) ? (double)(N - 1) : 1.0;
    if (J_total) *J_total = J0_obs + 0.5 * (double)(N - 1) * ww;
    for (int i = 0; i < N; ++i) w_out[i] = w[i] - alpha * g[i] / denom;
}

/* Observation vector of the DOMAIN cost (Eq. kinenergy normalised by the window length, R = I,
 * y = 0): h[t][cell][comp] = sqrt(dx dy / n_w) (u_c(t) - mean_t u_c) for the cell-centred
 * velocity of fluid cells at every window step (zero on solid cells), so that
 * J_domain = 1/2 ||h||^2.  Two passes: the window samples are stored first, then the window
 * means are subtracted.  h: n_window * nx * ny * 2 doubles. */
int orc_domain_observation(const orc_params *P, const double *u0, const double *v0, const double *fu,
                           const double *fv, int n_steps, int n_window, double *h)
{
    if (n_window < 1 || n_window > n_steps) return -1;
    orc_sim *s = orc_create(P);
    if (!s) return -2;
    orc_set_state(s, u0, v0, NULL);
    orc_set_face_forcing(s, fu, fv);
    int nx = s->nx, ny = s->ny;
    size_t nc = (size_t)nx * ny;
    orc_step(s, n_steps - n_window);
    for (int t = 0; t < n_window; ++t) {
        step_once(s);
        double *ht = h + (size_t)t * nc * 2;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t k = IC(s, i, j);
                ht[2 * k] = s->F[k] ? 0.5 * (s->u[IU(s, i, j)] + s->u[IU(s, i + 1, j)]) : 0.0;
                ht[2 * k + 1] = s->F[k] ? 0.5 * (s->v[IV(s, i, j)] + s->v[IV(s, i, j + 1)]) : 0.0;
            }
    }
    double wgt = sqrt(s->dx * s->dy / (double)n_window);
    for (size_t q = 0; q < 2 * nc; ++q) {
        double m = 0.0;
        for (int t = 0; t < n_window; ++t) m += h[(size_t)t * 2 * nc + q];
        m /= n_window;
        for (int t = 0; t < n_window; ++t) {
            double *x = &h[(size_t)t * 2 * nc + q];
            *x = (*x - m) * wgt;
        }
    }
    orc_destroy(s);
    return 0;
}

typedef struct {
    const orc_params *P;
    const double *region, *u0, *v0, *E, *w, *h0;
    int N, n_steps, n_window, n_ctrl;
    double eps;
    double *g, *ynorm2;
    int next;
    pthread_mutex_t lock;
} domain_job;

static void member_forcing_faces(const orc_params *P, const double *region, const double *E, const double *w,
                                 int N, int n_ctrl, double eps, int m, double *f, double *fu, double *fv)
{
    for (int r = 0; r < n_ctrl; ++r) {
        double acc = 0.0;
        for (int k = 0; k < N; ++k) acc += E[(size_t)k * n_ctrl + r] * w[k];
        if (m > 0) acc += eps * E[(size_t)(m - 1) * n_ctrl + r];
        f[r] = acc;
    }
    orc_control_to_faces(P, region, f, fu, fv);
}

static void *domain_worker(void *arg)
{
    domain_job *jb = (domain_job *)arg;
    const orc_params *P = jb->P;
    size_t nu_ = (size_t)(P->nx + 1) * P->ny, nv_ = (size_t)P->nx * (P->ny + 1);
    size_t nobs = (size_t)jb->n_window * P->nx * P->ny * 2;
    double *f = (double *)xcalloc((size_t)jb->n_ctrl, sizeof(double));
    double *fu = (double *)xcalloc(nu_, sizeof(double)), *fv = (double *)xcalloc(nv_, sizeof(double));
    double *hi = (double *)xcalloc(nobs, sizeof(double));
    for (;;) {
        pthread_mutex_lock(&jb->lock);
        int m = ++jb->next;
        pthread_mutex_unlock(&jb->lock);
        if (m > jb->N) break;
        member_forcing_faces(P, jb->region, jb->E, jb->w, jb->N, jb->n_ctrl, jb->eps, m, f, fu, fv);
        orc_domain_observation(P, jb->u0, jb->v0, fu, fv, jb->n_steps, jb->n_window, hi);
        /* column i of Y by Eq. (fdapprox), contracted with Hq_0 - y = h0 (Eq. gradient_EnVar) */
        double acc = 0.0, yy = 0.0;
        for (size_t k = 0; k < nobs; ++k) {
            double yk = (hi[k] - jb->h0[k]) / jb->eps;
            acc += yk * jb->h0[k];
            yy += yk * yk;
        }
        jb->g[m - 1] = acc + (double)(jb->N - 1) * jb->w[m - 1];
        if (jb->ynorm2) jb->ynorm2[m - 1] = yy;
    }
    free(f); free(fu); free(fv); free(hi);
    return NULL;
}

/* Eq. (gradient_EnVar) for the DOMAIN observation operator, with every column of Y from
 * Eq. (fdapprox):  g_i = Y_i^T (Hq_0 - y) + (N-1) w_i,  Y_i = (h_i - h_0)/eps,  h_m the
 * observation vector of member m (orc_domain_observation).  ynorm2 (may be NULL): ||Y_i||^2.
 * For J_obs = 1/2 ||h||^2 this differs from the scalar form (J_i - J_0)/eps by exactly
 * (eps/2) ||Y_i||^2. */
int orc_envar_gradient_domain(const orc_params *P, const double *region, const double *u0, const double *v0,
                              int n_ctrl, int N, const double *E, const double *w, double eps, int n_steps,
                              int n_window, int nthreads, double *g, double *ynorm2)
{
    int ncc = orc_control_cells(P, region, NULL, NULL);
    if (n_ctrl != 2 * ncc || n_window < 1) return -1;
    size_t nu_ = (size_t)(P->nx + 1) * P->ny, nv_ = (size_t)P->nx * (P->ny + 1);
    size_t nobs = (size_t)n_window * P->nx * P->ny * 2;
    double *h0 = (double *)xcalloc(nobs, sizeof(double));
    double *f = (double *)xcalloc((size_t)n_ctrl, sizeof(double));
    double *fu = (double *)xcalloc(nu_, sizeof(double)), *fv = (double *)xcalloc(nv_, sizeof(double));
    member_forcing_faces(P, region, E, w, N, n_ctrl, eps, 0, f, fu, fv);
    orc_domain_observation(P, u0, v0, fu, fv, n_steps, n_window, h0);
    free(f); free(fu); free(fv);
    domain_job jb;
    jb.P = P; jb.region = region; jb.u0 = u0; jb.v0 = v0; jb.E = E; jb.w = w; jb.h0 = h0;
    jb.N = N; jb.n_steps = n_steps; jb.n_window = n_window; jb.n_ctrl = n_ctrl; jb.eps = eps;
    jb.g = g; jb.ynorm2 = ynorm2; jb.next = 0;
    pthread_mutex_init(&jb.lock, NULL);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > N) nthreads = N > 0 ? N : 1;
    pthread_t *th = (pthread_t *)xcalloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, domain_worker, &jb);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&jb.lock);
    free(h0);
    return 0;
}

/* ------------------------ reduced-space optimisers ---------------------- */
/* Sensor-space observation anomalies of Eq. (fdapprox): h_m = series_m - its window mean
 * (8 n_window observations, R = I, y = 0), Y[i] = (h_{i+1} - h_0)/eps, i = 0..N-1, stored
 * row-wise [N][nobs]; h0 receives h_0 (nobs). */
void orc_sensor_anomalies(int N, int n_window, const double *series, double eps, double *Y, double *h0)
{
    size_t nobs = (size_t)n_window * 8;
    double *h = (double *)xcalloc(nobs, sizeof(double));
    for (int m = 0; m <= N; ++m) {
        const double *sm = series + (size_t)m * nobs;
        double *dst = (m == 0) ? h0 : h;
        for (int c = 0; c < 8; ++c) {
            double mean = 0.0;
            for (int t = 0; t < n_window; ++t) mean += sm[(size_t)t * 8 + c];
            mean /= n_window;
            for (int t = 0; t < n_window; ++t) dst[(size_t)t * 8 + c] = sm[(size_t)t * 8 + c] - mean;
        }
        if (m == 0) continue;
        for (size_t k = 0; k < nobs; ++k) Y[(size_t)(m - 1) * nobs + k] = (h[k] - h0[k]) / eps;
    }
    free(h);
}

/* Dense Cholesky A = L L^T (lower, row-major n x n, in place); returns -1 if A is not positive
 * definite.  Then solve A x = b. */
static int cholesky(int n, double *A)
{
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(d > 0.0)) return -1;
        d = sqrt(d);
        A[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double a = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) a -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = a / d;
        }
    }
    return 0;
}
static void cholesky_solve(int n, const double *L, const double *b, double *x)
{
    for (int i = 0; i < n; ++i) {
        double a = b[i];
        for (int k = 0; k < i; ++k) a -= L[(size_t)i * n + k] * x[k];
        x[i] = a / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double a = x[i];
        for (int k = i + 1; k < n; ++k) a -= L[(size_t)k * n + i] * x[k];
        x[i] = a / L[(size_t)i * n + i];
    }
}

/* Gauss-Newton step of Sec. 3.3.1: H_GN = Y^T R^{-1} Y + (N-1) I (Eq. Hessian_EnVar, R = I),
 * g = Y^T (Hq_0 - y) + (N-1) w (Eq. gradient_EnVar, y = 0), dw = -H_GN^{-1} g (Eq. update_Newton),
 * w_out = w + alpha dw.  Y: [N][nobs]; H_out (may be NULL): H_GN, row-major N x N; g_out (may be
 * NULL): g.  Returns -1 if H_GN is not positive definite. */
int orc_gauss_newton_step(int N, int nobs, const double *Y, const double *h0, const double *w, double alpha,
                          double *w_out, double *H_out, double *g_out)
{
    double *H = (double *)xcalloc((size_t)N * N, sizeof(double));
    double *g = (double *)xcalloc((size_t)N, sizeof(double));
    double *dw = (double *)xcalloc((size_t)N, sizeof(double));
    for (int i = 0; i < N; ++i) {
        double gi = 0.0;
        for (size_t k = 0; k < (size_t)nobs; ++k) gi += Y[(size_t)i * nobs + k] * h0[k];
        g[i] = gi + (double)(N - 1) * w[i];
        for (int j = 0; j < N; ++j) {
            double a = 0.0;
            for (size_t k = 0; k < (size_t)nobs; ++k) a += Y[(size_t)i * nobs + k] * Y[(size_t)j * nobs + k];
            H[(size_t)i * N + j] = a + (i == j ? (double)(N - 1) : 0.0);
        }
    }
    if (H_out) memcpy(H_out, H, sizeof(double) * (size_t)N * N);
    if (g_out) memcpy(g_out, g, sizeof(double) * (size_t)N);
    int rc = cholesky(N, H);
    if (rc == 0) {
        cholesky_solve(N, H, g, dw);
        for (int i = 0; i < N; ++i) w_out[i] = w[i] - alpha * dw[i];
    }
    free(H); free(g); free(dw);
    return rc;
}

/* L-BFGS search direction of Sec. 3.3.1 (Eq. update_BFGS): p = -H g with H the limited-memory BFGS
 * inverse-Hessian approximation built from the m most recent pairs s_k = w_{k+1} - w_k,
 * y_k = g_{k+1} - g_k (oldest first, rows of S and Yh, [m][N]) on the initial matrix gamma I,
 * evaluated by the two-loop recursion (Nocedal and Wright, Numerical Optimization, Alg. 7.4). */
void orc_lbfgs_direction(int N, int m, const double *S, const double *Yh, const double *g, double gamma, double *p)
{
    double *q = (double *)xcalloc((size_t)N, sizeof(double));
    double *a = (double *)xcalloc((size_t)(m > 0 ? m : 1), sizeof(double));
    for (int i = 0; i < N; ++i) q[i] = g[i];
    for (int k = m - 1; k >= 0; --k) {
        const double *s = S + (size_t)k * N, *y = Yh + (size_t)k * N;
        double sy = 0.0, sq = 0.0;
        for (int i = 0; i < N; ++i) { sy += s[i] * y[i]; sq += s[i] * q[i]; }
        a[k] = sq / sy;
        for (int i = 0; i < N; ++i) q[i] -= a[k] * y[i];
    }
    for (int i = 0; i < N; ++i) q[i] *= gamma;
    for (int k = 0; k < m; ++k) {
        const double *s = S + (size_t)k * N, *y = Yh + (size_t)k * N;
        double sy = 0.0, yq = 0.0;
        for (int i = 0; i < N; ++i) { sy += s[i] * y[i]; yq += y[i] * q[i]; }
        double b = yq / sy;
        for (int i = 0; i < N; ++i) q[i] += s[i] * (a[k] - b);
    }
    for (int i = 0; i < N; ++i) p[i] = -q[i];
    free(q); free(a);
}

typedef struct {
    const orc_params *P;
    const double *region, *u0, *v0, *E, *w;
    int N, n_steps, n_window, cost_mode, n_ctrl;
    double eps;
    double *J;
    double *series;  /* [N+1][n_window][8] or NULL */
    int next;        /* shared work counter */
    pthread_mutex_t lock;
} envar_job;

static void *envar_worker(void *arg)
{
    envar_job *jb = (envar_job *)arg;
    const orc_params *P = jb->P;
    size_t nu_ = (size_t)(P->nx + 1) * P->ny, nv_ = (size_t)P->nx * (P->ny + 1);
    double *f = (double *)xcalloc((size_t)jb->n_ctrl, sizeof(double));
    double *fu = (double *)xcalloc(nu_, sizeof(double)), *fv = (double *)xcalloc(nv_, sizeof(double));
    for (;;) {
        pthread_mutex_lock(&jb->lock);
        int m = jb->next++;
        pthread_mutex_unlock(&jb->lock);
        if (m > jb->N) break;
        /* f_m = E w (+ eps E_m for perturbed members), Eq. (fdapprox) */
        for (int r = 0; r < jb->n_ctrl; ++r) {
            double acc = 0.0;
            for (int k = 0; k < jb->N; ++k) acc += jb->E[(size_t)k * jb->n_ctrl + r] * jb->w[k];
            if (m > 0) acc += jb->eps * jb->E[(size_t)(m - 1) * jb->n_ctrl + r];
            f[r] = acc;
        }
        orc_control_to_faces(P, jb->region, f, fu, fv);
        double jd, js;
        double *ser = jb->series ? jb->series + (size_t)m * jb->n_window * 8 : NULL;
        orc_member_run(P, jb->u0, jb->v0, fu, fv, jb->n_steps, jb->n_window, &jd, &js, ser, NULL, NULL, NULL, NULL);
        jb->J[m] = (jb->cost_mode == 1) ? js : jd;
    }
    free(f); free(fu); free(fv);
    return NULL;
}

/* The N+1 forward evaluations of Fig. (envar_loop) and the gradient.
 * E: n_ctrl x N column-major; w: N; J: N+1 (observation cost per member,
 * member 0 unperturbed); g: N; J_prior: scalar.  cost_mode 0 = DOMAIN,
 * 1 = SENSORS.  series (may be NULL): sensor samples [N+1][n_window][8]. */
int orc_envar_gradient(const orc_params *P, const double *region, const double *u0, const double *v0,
                       int n_ctrl, int N, const double *E, const double *w, double eps,
                       int n_steps, int n_window, int cost_mode, int nthreads,
                       double *J, double *g, double *J_prior, double *series)
{
    int ncc = orc_control_cells(P, region, NULL, NULL);
    if (n_ctrl != 2 * ncc) return -1;
    envar_job jb;
    jb.P = P; jb.region = region; jb.u0 = u0; jb.v0 = v0; jb.E = E; jb.w = w;
    jb.N = N; jb.n_steps = n_steps; jb.n_window = n_window; jb.cost_mode = cost_mode; jb.n_ctrl = n_ctrl;
    jb.eps = eps; jb.J = J; jb.series = series; jb.next = 0;
    pthread_mutex_init(&jb.lock, NULL);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > N + 1) nthreads = N + 1;
    pthread_t *th = (pthread_t *)xcalloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, envar_worker, &jb);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&jb.lock);
    orc_gradient_from_costs(N, J, w, eps, g, J_prior);
    return 0;
}

/* ------------------------------- adjoint ------------------------------- */
/* Discrete adjoint of the time stepper above (Sec. 3.2, Eq. adjoint_discrete and
 * Eq. gradient_forcing in their discrete form): the gradient of the DOMAIN observation cost with
 * respect to a steady face forcing F (a vector on the unknown faces).
 *
 * One step maps X^n = (u^n on unknown and outlet faces) and the stored tendency R^{n-1} to
 *   v      = u^n + dt (c1 R(X^n) + c0 R^{n-1}) + dt F                (unknown faces)
 *   u_b'   = C(X^n)     (convective outlet + uniform flux shift)
 *   u^{n+1} = v - G psi,  L psi = D(v, u_b')    (projection; the p^n term drops out of u^{n+1})
 * so with mu = adjoint of u^{n+1} on unknown faces and nu on outlet faces:
 *   psi'   = L^{-1} D_u mu,  wbar = mu - G psi',  ubbar = nu + D_b^T psi'  (D_b: outlet columns)
 * and the adjoint of u^n collects wbar, J_R^T Rbar with Rbar = dt c1 wbar + dt c0' wbar' (the
 * next step's AB2 use of R^n), C^T ubbar, and the cost gradient at the window samples.  The
 * forcing gradient is dJ/dF = sum_n dt wbar.  Tendency transposes are taken by reverse mode of
 * explicit_rhs on the ghost-padded arrays, then the adjoint of the ghost filling. */

/* adjoint of fill_ghosts: padded adjoints -> compact adjoints (accumulated) */
static void fill_ghosts_adjoint(orc_sim *s, double *Ub, double *Vb, double *lu, double *lv)
{
    int nx = s->nx, ny = s->ny;
#define UB(i, j) (Ub[(size_t)((j) + 1) * (size_t)(nx + 3) + (size_t)((i) + 1)])
#define VB(i, j) (Vb[(size_t)((j) + 1) * (size_t)(nx + 2) + (size_t)((i) + 1)])
    /* reverse order of fill_ghosts: y edges, x edges, buried faces, interior copy */
    for (int i = nx; i >= -1; --i) {
        if (s->P.bc_y == 1) {
            VB(i, 1) += VB(i, ny + 1); VB(i, ny + 1) = 0.0;
            VB(i, ny - 1) += VB(i, -1); VB(i, -1) = 0.0;
            VB(i, 0) += VB(i, ny); VB(i, ny) = 0.0;
        } else {
            VB(i, -1) = 0.0; VB(i, ny + 1) = 0.0;
        }
    }
    for (int i = nx + 1; i >= -1; --i) {
        if (s->P.bc_y == 1) {
            UB(i, 0) += UB(i, ny); UB(i, ny) = 0.0;
            UB(i, ny - 1) += UB(i, -1); UB(i, -1) = 0.0;
        } else if (s->P.bc_y == 2) {
            UB(i, ny - 1) -= UB(i, ny); UB(i, ny) = 0.0;
            UB(i, 0) -= UB(i, -1); UB(i, -1) = 0.0;
        } else {
            UB(i, ny - 1) += UB(i, ny); UB(i, ny) = 0.0;
            UB(i, 0) -= UB(i, -1); UB(i, -1) = 0.0;
        }
    }
    for (int j = ny; j >= 0; --j) {
        if (s->P.bc_x == 1) {
            VB(0, j) += VB(nx, j); VB(nx, j) = 0.0;
            VB(nx - 1, j) += VB(-1, j); VB(-1, j) = 0.0;
        } else {
            VB(nx - 1, j) += VB(nx, j); VB(nx, j) = 0.0;
            VB(0, j) -= VB(-1, j); VB(-1, j) = 0.0;
        }
    }
    for (int j = ny - 1; j >= 0; --j) {
        if (s->P.bc_x == 1) {
            UB(1, j) += UB(nx + 1, j); UB(nx + 1, j) = 0.0;
            UB(nx - 1, j) += UB(-1, j); UB(-1, j) = 0.0;
            UB(0, j) += UB(nx, j); UB(nx, j) = 0.0;
        } else {
            UB(-1, j) = 0.0; UB(nx + 1, j) = 0.0;
        }
    }
    for (int j = ny; j >= 0; --j)
        for (int i = nx - 1; i >= 0; --i) {
            if (s->vk[IV(s, i, j)] != FK_SOLID) continue;
            int rt = (i + 1 < nx) && s->vk[IV(s, i + 1, j)] == FK_UNKNOWN;
            int lt = (i - 1 >= 0) && s->vk[IV(s, i - 1, j)] == FK_UNKNOWN;
            if (rt) lv[IV(s, i + 1, j)] -= VB(i, j);
            else if (lt) lv[IV(s, i - 1, j)] -= VB(i, j);
            VB(i, j) = 0.0;
        }
    for (int j = ny - 1; j >= 0; --j)
        for (int i = nx; i >= 0; --i) {
            if (s->uk[IU(s, i, j)] != FK_SOLID) continue;
            int up = (j + 1 < ny) && s->uk[IU(s, i, j + 1)] == FK_UNKNOWN;
            int dn = (j - 1 >= 0) && s->uk[IU(s, i, j - 1)] == FK_UNKNOWN;
            if (up) lu[IU(s, i, j + 1)] += lower_wall_sign(s, i) * UB(i, j);
            else if (dn) lu[IU(s, i, j - 1)] -= UB(i, j);
            UB(i, j) = 0.0;
        }
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) lu[IU(s, i, j)] += UB(i, j);
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) lv[IV(s, i, j)] += VB(i, j);
#undef UB
#undef VB
}

/* lu, lv += (dR/du)^T Rbu, (dR/dv)^T Rbv at the state held in s (reverse mode of explicit_rhs) */
static void explicit_rhs_adjoint(orc_sim *s, const double *Rbu, const double *Rbv, double *lu, double *lv)
{
    int nx = s->nx, ny = s->ny;
    double dx = s->dx, dy = s->dy, nu = s->nu;
    int adv = s->P.advection;
    size_t nug = (size_t)(nx + 3) * (ny + 2), nvg = (size_t)(nx + 2) * (ny + 3);
    double *Ub = (double *)xcalloc(nug, sizeof(double)), *Vb = (double *)xcalloc(nvg, sizeof(double));
#define UB(i, j) (Ub[(size_t)((j) + 1) * (size_t)(nx + 3) + (size_t)((i) + 1)])
#define VB(i, j) (Vb[(size_t)((j) + 1) * (size_t)(nx + 2) + (size_t)((i) + 1)])
    fill_ghosts(s, s->u, s->v);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            size_t k = IU(s, i, j);
            if (s->uk[k] != FK_UNKNOWN) continue;
            double rb = Rbu[k];
            if (rb == 0.0) continue;
            double uc = UG(s, i, j), ue = UG(s, i + 1, j), uw = UG(s, i - 1, j);
            double un = UG(s, i, j + 1), us = UG(s, i, j - 1);
            /* diffusion */
            double cxx = nu / (dx * dx), cyy = nu / (dy * dy);
            UB(i, j) += rb * (-2.0 * cxx - 2.0 * cyy);
            UB(i + 1, j) += rb * cxx; UB(i - 1, j) += rb * cxx;
            UB(i, j + 1) += rb * cyy; UB(i, j - 1) += rb * cyy;
            if (adv) {
                /* R = -A: A = (fe^2 - fw^2)/dx + (un_c vn_c - us_c vs_c)/dy */
                double fe = 0.5 * (uc + ue), fw = 0.5 * (uw + uc);
                double un_c = 0.5 * (uc + un), vn_c = 0.5 * (VG(s, i - 1, j + 1) + VG(s, i, j + 1));
                double us_c = 0.5 * (us + uc), vs_c = 0.5 * (VG(s, i - 1, j) + VG(s, i, j));
                double a = -rb;   /* adjoint of A */
                double bfe = a * 2.0 * fe / dx, bfw = -a * 2.0 * fw / dx;
                double bun = a * vn_c / dy, bvn = a * un_c / dy;
                double bus = -a * vs_c / dy, bvs = -a * us_c / dy;
                UB(i, j) += 0.5 * bfe + 0.5 * bfw + 0.5 * bun + 0.5 * bus;
                UB(i + 1, j) += 0.5 * bfe;
                UB(i - 1, j) += 0.5 * bfw;
                UB(i, j + 1) += 0.5 * bun;
                UB(i, j - 1) += 0.5 * bus;
                VB(i - 1, j + 1) += 0.5 * bvn; VB(i, j + 1) += 0.5 * bvn;
                VB(i - 1, j) += 0.5 * bvs; VB(i, j) += 0.5 * bvs;
            }
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = IV(s, i, j);
            if (s->vk[k] != FK_UNKNOWN) continue;
            double rb = Rbv[k];
            if (rb == 0.0) continue;
            double vc = VG(s, i, j), ve = VG(s, i + 1, j), vw = VG(s, i - 1, j);
            double vn = VG(s, i, j + 1), vs = VG(s, i, j - 1);
            double cxx = nu / (dx * dx), cyy = nu / (dy * dy);
            VB(i, j) += rb * (-2.0 * cxx - 2.0 * cyy);
            VB(i + 1, j) += rb * cxx; VB(i - 1, j) += rb * cxx;
            VB(i, j + 1) += rb * cyy; VB(i, j - 1) += rb * cyy;
            if (adv) {
                /* A = (ue_c ve_c - uw_c vw_c)/dx + (fn^2 - fs^2)/dy */
                double ue_c = 0.5 * (UG(s, i + 1, j - 1) + UG(s, i + 1, j)), ve_c = 0.5 * (vc + ve);
                double uw_c = 0.5 * (UG(s, i, j - 1) + UG(s, i, j)), vw_c = 0.5 * (vw + vc);
                double fn = 0.5 * (vc + vn), fs = 0.5 * (vs + vc);
                double a = -rb;
                double bue = a * ve_c / dx, bve = a * ue_c / dx;
                double buw = -a * vw_c / dx, bvw = -a * uw_c / dx;
                double bfn = a * 2.0 * fn / dy, bfs = -a * 2.0 * fs / dy;
                UB(i + 1, j - 1) += 0.5 * bue; UB(i + 1, j) += 0.5 * bue;
                UB(i, j - 1) += 0.5 * buw; UB(i, j) += 0.5 * buw;
                VB(i, j) += 0.5 * bve + 0.5 * bvw + 0.5 * bfn + 0.5 * bfs;
                VB(i + 1, j) += 0.5 * bve;
                VB(i - 1, j) += 0.5 * bvw;
                VB(i, j + 1) += 0.5 * bfn;
                VB(i, j - 1) += 0.5 * bfs;
            }
        }
#undef UB
#undef VB
    fill_ghosts_adjoint(s, Ub, Vb, lu, lv);
    free(Ub); free(Vb);
}

/* Adjoint gradient of the DOMAIN cost with respect to the face forcing (fu, fv), and the cost.
 * gu / gv: dJ/dF on unknown faces (zero elsewhere).  Stores all n_steps + 1 states. */
int orc_adjoint_gradient(const orc_params *P, const double *u0, const double *v0, const double *fu, const double *fv,
                         int n_steps, int n_window, double *J_out, double *gu, double *gv)
{
    if (P->bc_x != 0 || n_window < 1 || n_window > n_steps) return -1;
    orc_sim *s = orc_create(P);
    if (!s) return -2;
    int nx = s->nx, ny = s->ny;
    size_t nc = (size_t)nx * ny, nu_ = (size_t)(nx + 1) * ny, nv_ = (size_t)nx * (ny + 1);
    double *U = (double *)xcalloc(nu_ * (size_t)(n_steps + 1), sizeof(double));
    double *V = (double *)xcalloc(nv_ * (size_t)(n_steps + 1), sizeof(double));
    orc_set_state(s, u0, v0, NULL);
    orc_set_face_forcing(s, fu, fv);
    memcpy(U, s->u, nu_ * sizeof(double));
    memcpy(V, s->v, nv_ * sizeof(double));
    for (int n = 0; n < n_steps; ++n) {
        step_once(s);
        memcpy(U + nu_ * (size_t)(n + 1), s->u, nu_ * sizeof(double));
        memcpy(V + nv_ * (size_t)(n + 1), s->v, nv_ * sizeof(double));
    }
    /* window means and the cost (two-pass on the stored samples) */
    int k0 = n_steps - n_window + 1;
    double *mu = (double *)xcalloc(nc, sizeof(double)), *mv = (double *)xcalloc(nc, sizeof(double));
    for (int k = k0; k <= n_steps; ++k) {
        const double *u = U + nu_ * (size_t)k, *v = V + nv_ * (size_t)k;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IC(s, i, j);
                if (!s->F[c]) continue;
                mu[c] += 0.5 * (u[IU(s, i, j)] + u[IU(s, i + 1, j)]);
                mv[c] += 0.5 * (v[IV(s, i, j)] + v[IV(s, i, j + 1)]);
            }
    }
    for (size_t c = 0; c < nc; ++c) { mu[c] /= n_window; mv[c] /= n_window; }
    double J = 0.0, wgt = s->dx * s->dy / (double)n_window;
    for (int k = k0; k <= n_steps; ++k) {
        const double *u = U + nu_ * (size_t)k, *v = V + nv_ * (size_t)k;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IC(s, i, j);
                if (!s->F[c]) continue;
                double a = 0.5 * (u[IU(s, i, j)] + u[IU(s, i + 1, j)]) - mu[c];
                double b = 0.5 * (v[IV(s, i, j)] + v[IV(s, i, j + 1)]) - mv[c];
                J += 0.5 * wgt * (a * a + b * b);
            }
    }
    /* reverse sweep */
    double *lu = (double *)xcalloc(nu_, sizeof(double)), *lv = (double *)xcalloc(nv_, sizeof(double));
    double *wu = (double *)xcalloc(nu_, sizeof(double)), *wv = (double *)xcalloc(nv_, sizeof(double));
    double *cu = (double *)xcalloc(nu_, sizeof(double)), *cv = (double *)xcalloc(nv_, sizeof(double));
    double *Rbu = (double *)xcalloc(nu_, sizeof(double)), *Rbv = (double *)xcalloc(nv_, sizeof(double));
    double *psi = (double *)xcalloc(nc, sizeof(double)), *rhs = (double *)xcalloc(nc, sizeof(double));
    double *ubb = (double *)xcalloc((size_t)ny, sizeof(double));
    double dt = s->P.dt, kap = dt * s->P.conv_speed / s->dx;
    for (size_t k = 0; k < nu_; ++k) gu[k] = 0.0;
    for (size_t k = 0; k < nv_; ++k) gv[k] = 0.0;
    int nout = 0;
    for (int j = 0; j < ny; ++j) nout += (s->uk[IU(s, nx, j)] == FK_OUTLET);
    for (int n = n_steps; n >= 0; --n) {
        /* cost gradient at sample n: d/du_face of sum_c wgt/2 |u_c - mean|^2 */
        if (n >= k0) {
            const double *u = U + nu_ * (size_t)n, *v = V + nv_ * (size_t)n;
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t c = IC(s, i, j);
                    if (!s->F[c]) continue;
                    double a = 0.5 * (u[IU(s, i, j)] + u[IU(s, i + 1, j)]) - mu[c];
                    double b = 0.5 * (v[IV(s, i, j)] + v[IV(s, i, j + 1)]) - mv[c];
                    lu[IU(s, i, j)] += 0.5 * wgt * a; lu[IU(s, i + 1, j)] += 0.5 * wgt * a;
                    lv[IV(s, i, j)] += 0.5 * wgt * b; lv[IV(s, i, j + 1)] += 0.5 * wgt * b;
                }
        }
        if (n == 0) break;
        /* reverse the step (n-1) -> n */
        int m = n - 1;
        double c1 = (m == 0) ? 1.0 : 1.5, c0 = (m == 0) ? 0.0 : -0.5;
        /* psi = L^{-1} D_u mu  <=>  (-L) psi = -D_u mu (mu on unknown faces only) */
        for (size_t k = 0; k < nu_; ++k) wu[k] = (s->uk[k] == FK_UNKNOWN) ? lu[k] : 0.0;
        for (size_t k = 0; k < nv_; ++k) wv[k] = (s->vk[k] == FK_UNKNOWN) ? lv[k] : 0.0;
        divergence(s, wu, wv, -1.0, rhs);
        remove_mean(s, rhs);
        for (size_t k = 0; k < nc; ++k) psi[k] = 0.0;
        pcg_solve(s, rhs, psi);
        /* wbar = mu - G psi (unknown faces) */
        grad_correct(s, wu, wv, psi, 1.0);
        /* outlet: ubbar_j = nu_j + psi(nx-1, j)/dx */
        for (int j = 0; j < ny; ++j)
            ubb[j] = (s->uk[IU(s, nx, j)] == FK_OUTLET) ? lu[IU(s, nx, j)] + psi[IC(s, nx - 1, j)] / s->dx : 0.0;
        /* Rbar = dt c1 wbar + carry; carry = dt c0 wbar; forcing gradient */
        for (size_t k = 0; k < nu_; ++k) {
            Rbu[k] = dt * c1 * wu[k] + cu[k];
            cu[k] = dt * c0 * wu[k];
            gu[k] += dt * wu[k];
        }
        for (size_t k = 0; k < nv_; ++k) {
            Rbv[k] = dt * c1 * wv[k] + cv[k];
            cv[k] = dt * c0 * wv[k];
            gv[k] += dt * wv[k];
        }
        /* lambda^m = wbar + J_R(X^m)^T Rbar + C^T ubbar */
        for (size_t k = 0; k < nu_; ++k) lu[k] = wu[k];
        for (size_t k = 0; k < nv_; ++k) lv[k] = wv[k];
        memcpy(s->u, U + nu_ * (size_t)m, nu_ * sizeof(double));
        memcpy(s->v, V + nv_ * (size_t)m, nv_ * sizeof(double));
        explicit_rhs_adjoint(s, Rbu, Rbv, lu, lv);
        /* C: ub_j = (1-kap) u_nx,j + kap u_nx-1,j + shift, shift = (Qin/dy - sum_k ub'_k)/nout */
        double sb = 0.0;
        for (int j = 0; j < ny; ++j) sb += ubb[j];
        for (int j = 0; j < ny; ++j) {
            if (s->uk[IU(s, nx, j)] != FK_OUTLET) continue;
            double bp = ubb[j] - sb / nout;
            lu[IU(s, nx, j)] += (1.0 - kap) * bp;
            lu[IU(s, nx - 1, j)] += kap * bp;
        }
    }
    if (J_out) *J_out = J;
    free(U); free(V); free(mu); free(mv); free(lu); free(lv); free(wu); free(wv); free(cu); free(cv);
    free(Rbu); free(Rbv); free(psi); free(rhs); free(ubb);
    orc_destroy(s);
    return 0;
}

/* Control-space gradient: g[c] = P^T dJ/dF, the transpose of orc_control_to_faces. */
void orc_faces_to_control(const orc_params *P, const double *region, const double *gu, const double *gv, double *g)
{
    int nx = P->nx, ny = P->ny;
    int nc = orc_control_cells(P, region, NULL, NULL);
    int *ci = (int *)xcalloc((size_t)nc, sizeof(int)), *cj = (int *)xcalloc((size_t)nc, sizeof(int));
    orc_control_cells(P, region, ci, cj);
    orc_sim *s = orc_create(P);
    for (int q = 0; q < nc; ++q) {
        int i = ci[q], j = cj[q];
        double ax = 0.0, ay = 0.0;
        for (int f = i; f <= i + 1; ++f) {
            size_t k = (size_t)j * (nx + 1) + f;
            if (s->uk[k] == FK_UNKNOWN) ax += 0.5 * gu[k];
        }
        for (int f = j; f <= j + 1; ++f) {
            size_t k = (size_t)f * nx + i;
            if (s->vk[k] == FK_UNKNOWN) ay += 0.5 * gv[k];
        }
        g[q] = ax;
        g[nc + q] = ay;
    }
    orc_destroy(s);
    free(ci); free(cj);
    (void)ny;
}
