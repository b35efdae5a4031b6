// k_adjoint.cu -- discrete adjoint of the FP64 time stepper (Sec. 3.2, Eq. adjoint_discrete and
// Eq. gradient_forcing in their discrete form): the reference gradient of the DOMAIN cost with
// respect to the steady forcing, member slot 0.
//
// Forward step n -> n+1 (k_flow.cu): v = u^n + dt (c1 R(X^n) + c0 R^{n-1}) + dt F on unknown faces,
// u_b = C(X^n) on outlet faces (convective update + uniform flux shift), u^{n+1} = v - G psi with
// L psi = D(v, u_b); p^n drops out of u^{n+1}.  Reverse step, given lambda = adjoint of X^{n+1}:
//   (1) k_adj_rhs:   b = -dx dy D_u(mu)  (mu = lambda on unknown faces; FV form of L psi = D_u mu),
//                    scaled to max|b| = 1 (the scale s is kept on the device)
//   (2) the FP64 multigrid-preconditioned CG of k_poisson.cu solves A x = b / s; psi = s x
//   (3) k_adj_post:  wbar = mu - G psi;  u_b-bar = nu + psi(nx-1)/dx;  Rbar = dt c1 wbar + carry;
//                    carry = dt c0 wbar;  dJ/dF += dt wbar;  lambda <- wbar (0 off unknown faces)
//   (4) k_adj_tend:  lambda += J_R(X^n)^T Rbar  (reverse mode of the stencil, same mirror rules as
//                    the forward, scattered with FP64 atomics)
//   (5) k_adj_outlet: lambda += C^T u_b-bar
//   (6) k_adj_cost:  lambda += dJ/dX^n at window samples (dx dy / n_w) H^T (u_c - mean u_c)
#include "envar_internal.cuh"
#include "../../include/envar.h"

namespace envar {

// b = -dx dy D_u(mu), and max |b| into *mx (as the bit pattern of a non-negative double, whose
// integer order is its numeric order)
__global__ void k_adj_rhs(Grid g, const double *__restrict__ lu, const double *__restrict__ lv, double *__restrict__ b,
                          unsigned long long *mx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    double r = 0.0;
    if (i < g.nx && j < g.ny) {
        const long long c = (long long)j * g.P + i;
        if (g.fluid[c]) {
            const double mE = (g.uk[c + 1] == FK_UNK) ? lu[c + 1] : 0.0, mW = (g.uk[c] == FK_UNK) ? lu[c] : 0.0;
            const double mN = (g.vk[c + g.P] == FK_UNK) ? lv[c + g.P] : 0.0, mS = (g.vk[c] == FK_UNK) ? lv[c] : 0.0;
            r = -(g.dy * (mE - mW) + g.dx * (mN - mS));
        }
        b[c] = r;
    }
    const double m = block_reduce(fabs(r), true);
    if (threadIdx.x == 0 && threadIdx.y == 0 && m > 0.0) atomicMax(mx, (unsigned long long)__double_as_longlong(m));
}

// b <- b / max|b|: the solve then runs on a right-hand side of unit size, so one relative stopping
// tolerance serves every reverse step whatever the size of the adjoint
__global__ void k_adj_scale(Grid g, double *__restrict__ b, const unsigned long long *mx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const double s = __longlong_as_double((long long)*mx);
    const long long c = (long long)j * g.P + i;
    b[c] = (s > 0.0) ? b[c] / s : 0.0;
}

// start of a reverse step: clear the solve's convergence flags and the scale
__global__ void k_adj_begin(MemberCtl *ctl, unsigned long long *mx)
{
    ctl[0].outer_done = 0;
    ctl[0].inner_done = 0;
    *mx = 0ULL;
}

// working state restored to forward state k: the next forward step is step k + 1
__global__ void k_adj_set_step(MemberCtl *ctl, int k) { ctl[0].step = k; }

__global__ void k_adj_post(Grid g, double *__restrict__ lu, double *__restrict__ lv, const double *__restrict__ x,
                           const unsigned long long *mx, const MemberRed *red, double res_tol, MemberCtl *ctl,
                           double *__restrict__ ubb, double *__restrict__ Rbu, double *__restrict__ Rbv,
                           double *__restrict__ cu, double *__restrict__ cv, double *__restrict__ gu,
                           double *__restrict__ gv, double c1, double c0)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i == 0 && j == 0 && !(red[0].val[RS_RMAX] <= res_tol)) atomicOr(&ctl[0].status, ENVAR_ST_ADJOINT);
    if (i > g.nx || j > g.ny) return;
    const long long c = (long long)j * g.P + i;
    const double dt = g.dt;
    const double sc = __longlong_as_double((long long)*mx);   // psi = sc * x
    auto psi = [&](long long cc) { return sc * x[cc]; };
    if (j < g.ny) {
        const uint8_t k = g.uk[c];
        double w = 0.0;
        if (k == FK_UNK) w = lu[c] - (psi(c) - psi(c - 1)) / g.dx;
        if (k == FK_OUTLET) ubb[j] = lu[c] + psi(c - 1) / g.dx;
        else if (i == g.nx) ubb[j] = 0.0;
        Rbu[c] = dt * c1 * w + cu[c];
        cu[c] = dt * c0 * w;
        gu[c] += dt * w;
        lu[c] = w;
    }
    if (i < g.nx) {
        double w = 0.0;
        if (g.vk[c] == FK_UNK) w = lv[c] - (psi(c) - psi(c - g.P)) / g.dy;
        Rbv[c] = dt * c1 * w + cv[c];
        cv[c] = dt * c0 * w;
        gv[c] += dt * w;
        lv[c] = w;
    }
}

__global__ void k_adj_tend(Grid g, const double *__restrict__ u, const double *__restrict__ v,
                           const double *__restrict__ Rbu, const double *__restrict__ Rbv, double *lu, double *lv)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > g.nx || j > g.ny) return;
    const long long c = (long long)j * g.P + i;
    const int P = g.P;
    const double i4dx = 0.25 / g.dx, i4dy = 0.25 / g.dy;
    const double nx2 = g.nu / (g.dx * g.dx), ny2 = g.nu / (g.dy * g.dy);
    if (j < g.ny && g.uk[c] == FK_UNK) {
        const double rb = Rbu[c];
        if (rb != 0.0) {
            const double uc = u[c], ue = u[c + 1], uw = u[c - 1];
            // north / south neighbours: array value, or the mirror of uc (solid face, bottom wall),
            // or uc itself (free-slip top)
            long long cn = c + P, cs = c - P;
            double sn = 1.0, ss = 1.0;
            if (j + 1 == g.ny) { cn = c; sn = 1.0; }
            else if (g.uk[c + P] == FK_SOLID) { cn = c; sn = -1.0; }
            else if (g.uk[c + P] == FK_SLIP) { cn = c; sn = 1.0; }
            if (j == 0) { cs = c; ss = -1.0; }
            else if (g.uk[c - P] == FK_SOLID) { cs = c; ss = -1.0; }
            else if (g.uk[c - P] == FK_SLIP) { cs = c; ss = 1.0; }
            const double un = sn * u[cn], us = ss * u[cs];
            const double vn = v[c + P - 1] + v[c + P], vs = v[c - 1] + v[c];
            const double dUc = -(2.0 * (uc + ue) - 2.0 * (uw + uc)) * i4dx - (vn - vs) * i4dy - 2.0 * nx2 - 2.0 * ny2;
            const double dUe = -2.0 * (uc + ue) * i4dx + nx2;
            const double dUw = 2.0 * (uw + uc) * i4dx + nx2;
            const double dUn = -vn * i4dy + ny2;
            const double dUs = vs * i4dy + ny2;
            const double dVn = -(uc + un) * i4dy, dVs = (us + uc) * i4dy;
            atomicAdd(&lu[c], rb * dUc);
            atomicAdd(&lu[c + 1], rb * dUe);
            atomicAdd(&lu[c - 1], rb * dUw);
            atomicAdd(&lu[cn], sn * rb * dUn);
            atomicAdd(&lu[cs], ss * rb * dUs);
            atomicAdd(&lv[c + P - 1], rb * dVn);
            atomicAdd(&lv[c + P], rb * dVn);
            atomicAdd(&lv[c - 1], rb * dVs);
            atomicAdd(&lv[c], rb * dVs);
        }
    }
    if (i < g.nx && g.vk[c] == FK_UNK) {
        const double rb = Rbv[c];
        if (rb != 0.0) {
            const double vc = v[c], vn = v[c + P], vs = v[c - P];
            long long ce = c + 1, cw = c - 1;
            double se = 1.0, sw = 1.0;
            if (i + 1 == g.nx) { ce = c; se = 1.0; } else if (g.vk[c + 1] == FK_SOLID) { ce = c; se = -1.0; }
            if (i == 0) { cw = c; sw = -1.0; } else if (g.vk[c - 1] == FK_SOLID) { cw = c; sw = -1.0; }
            const double ve = se * v[ce], vw = sw * v[cw];
            const double ue = u[c - P + 1] + u[c + 1], uw = u[c - P] + u[c];
            const double dVc = -(ue - uw) * i4dx - (2.0 * (vc + vn) - 2.0 * (vs + vc)) * i4dy - 2.0 * nx2 - 2.0 * ny2;
            const double dVe = -ue * i4dx + nx2;
            const double dVw = uw * i4dx + nx2;
            const double dVn = -2.0 * (vc + vn) * i4dy + ny2;
            const double dVs = 2.0 * (vs + vc) * i4dy + ny2;
            const double dUe = -(vc + ve) * i4dx, dUw = (vw + vc) * i4dx;
            atomicAdd(&lv[c], rb * dVc);
            atomicAdd(&lv[ce], se * rb * dVe);
            atomicAdd(&lv[cw], sw * rb * dVw);
            atomicAdd(&lv[c + P], rb * dVn);
            atomicAdd(&lv[c - P], rb * dVs);
            atomicAdd(&lu[c - P + 1], rb * dUe);
            atomicAdd(&lu[c + 1], rb * dUe);
            atomicAdd(&lu[c - P], rb * dUw);
            atomicAdd(&lu[c], rb * dUw);
        }
    }
}

__global__ void k_adj_outlet(Grid g, const double *__restrict__ ubb, double *lu)
{
    double sb = 0.0, nout = 0.0;
    for (int j = threadIdx.x; j < g.ny; j += blockDim.x) {
        if (g.uk[(long long)j * g.P + g.nx] == FK_OUTLET) { sb += ubb[j]; nout += 1.0; }
    }
    sb = block_reduce(sb, false);
    nout = block_reduce(nout, false);
    const double kap = g.dt * g.conv_speed / g.dx;
    for (int j = threadIdx.x; j < g.ny; j += blockDim.x) {
        const long long c = (long long)j * g.P + g.nx;
        if (g.uk[c] != FK_OUTLET) continue;
        const double bp = ubb[j] - sb / nout;
        lu[c] += (1.0 - kap) * bp;
        lu[c - 1] += kap * bp;
    }
}

__global__ void k_adj_cost(Grid g, const double *__restrict__ u, const double *__restrict__ v,
                           const double *__restrict__ mu, const double *__restrict__ mv, double wgt, double *lu,
                           double *lv)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > g.nx || j > g.ny) return;
    const long long c = (long long)j * g.P + i;
    auto du_cell = [&](long long cc) { return 0.5 * (u[cc] + u[cc + 1]) - mu[cc]; };
    auto dv_cell = [&](long long cc) { return 0.5 * (v[cc] + v[cc + g.P]) - mv[cc]; };
    if (j < g.ny) {
        double a = 0.0;
        if (i >= 1 && g.fluid[c - 1]) a += du_cell(c - 1);
        if (i < g.nx && g.fluid[c]) a += du_cell(c);
        lu[c] += 0.5 * wgt * a;
    }
    if (i < g.nx) {
        double b = 0.0;
        if (j >= 1 && g.fluid[c - g.P]) b += dv_cell(c - g.P);
        if (j < g.ny && g.fluid[c]) b += dv_cell(c);
        lv[c] += 0.5 * wgt * b;
    }
}

// control-space gradient g[c] = P^T dJ/dF: each control cell collects half of its unknown faces
__global__ void k_faces_to_control(Grid g, int ncc, const int *__restrict__ cidx, const double *__restrict__ gu,
                                   const double *__restrict__ gv, double *__restrict__ out)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < ncc; q += gridDim.x * blockDim.x) {
        const int r = cidx[q];
        const int i = g.ia + r % g.nrx, j = g.ja + r / g.nrx;
        const long long c = (long long)j * g.P + i;
        double ax = 0.0, ay = 0.0;
        if (g.uk[c] == FK_UNK) ax += 0.5 * gu[c];
        if (g.uk[c + 1] == FK_UNK) ax += 0.5 * gu[c + 1];
        if (g.vk[c] == FK_UNK) ay += 0.5 * gv[c];
        if (g.vk[c + g.P] == FK_UNK) ay += 0.5 * gv[c + g.P];
        out[q] = ax;
        out[ncc + q] = ay;
    }
}

void launch_adj_rhs(const Grid &g, const double *lu, const double *lv, double *b, unsigned long long *mx,
                    MemberCtl *ctl, cudaStream_t st)
{
    dim3 blk(32, 8), grd(cdiv(g.nx, 32), cdiv(g.ny, 8), 1);
    k_adj_begin<<<1, 1, 0, st>>>(ctl, mx);
    k_adj_rhs<<<grd, blk, 0, st>>>(g, lu, lv, b, mx);
    k_adj_scale<<<grd, blk, 0, st>>>(g, b, mx);
    count_launches(3);
}
void launch_adj_set_step(MemberCtl *ctl, int k, cudaStream_t st)
{
    k_adj_set_step<<<1, 1, 0, st>>>(ctl, k);
    count_launches(1);
}
void launch_adj_post(const Grid &g, double *lu, double *lv, const double *x, const unsigned long long *mx,
                     const MemberRed *red, double res_tol, MemberCtl *ctl, double *ubb, double *Rbu, double *Rbv,
                     double *cu, double *cv, double *gu, double *gv, double c1, double c0, cudaStream_t st)
{
    dim3 blk(32, 8), grd(cdiv(g.nx + 1, 32), cdiv(g.ny + 1, 8), 1);
    k_adj_post<<<grd, blk, 0, st>>>(g, lu, lv, x, mx, red, res_tol, ctl, ubb, Rbu, Rbv, cu, cv, gu, gv, c1, c0);
    count_launches(1);
}
void launch_adj_tend(const Grid &g, const double *u, const double *v, const double *Rbu, const double *Rbv, double *lu,
                     double *lv, cudaStream_t st)
{
    dim3 blk(32, 8), grd(cdiv(g.nx + 1, 32), cdiv(g.ny + 1, 8), 1);
    k_adj_tend<<<grd, blk, 0, st>>>(g, u, v, Rbu, Rbv, lu, lv);
    count_launches(1);
}
void launch_adj_outlet(const Grid &g, const double *ubb, double *lu, cudaStream_t st)
{
    k_adj_outlet<<<1, 256, 0, st>>>(g, ubb, lu);
    count_launches(1);
}
void launch_adj_cost(const Grid &g, const double *u, const double *v, const double *mu, const double *mv, double wgt,
                     double *lu, double *lv, cudaStream_t st)
{
    dim3 blk(32, 8), grd(cdiv(g.nx + 1, 32), cdiv(g.ny + 1, 8), 1);
    k_adj_cost<<<grd, blk, 0, st>>>(g, u, v, mu, mv, wgt, lu, lv);
    count_launches(1);
}
void launch_faces_to_control(const Grid &g, int ncc, const int *cidx, const double *gu, const double *gv, double *out,
                             cudaStream_t st)
{
    k_faces_to_control<<<cdiv(ncc, 256), 256, 0, st>>>(g, ncc, cidx, gu, gv, out);
    count_launches(1);
}

} // namespace envar
