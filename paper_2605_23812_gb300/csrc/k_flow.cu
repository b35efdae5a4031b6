// k_flow.cu -- time-stepper kernels of the forced Navier-Stokes solver (Sec. 2, Eq. forced_NS /
// Eq. discrete_NS) on the staggered MAC grid, batched over ensemble members (blockIdx.z).
//
// Step n -> n+1 (explicit AB2 on advection + diffusion, steady forcing P f, incremental projection):
//   k_outflow : convective outlet u_b^{n+1} = u_b^n - dt Uc (u_b^n - u_{nx-1}^n)/dx, then a uniform
//               shift so the outflow flux equals the inflow flux (the Neumann Poisson problem is
//               then compatible).  Advances the member's step counter.
//   k_predict : R^n = -div(u u) + nu lap(u)  (central, divergence form) in TR precision;
//               u* = u^n + dt (c1 R^n + c0 R^{n-1}) + dt P f - dt G p^n   (c = (1,0) on step 1, else (3/2,-1/2))
//   k_rhs     : b = -(dx dy / dt) D u*            (finite-volume form of L dp = D u*/dt)
//   [pressure solve A dp = b, k_poisson.cu]
//   k_correct : u^{n+1} = u* - dt G dp,  p^{n+1} = p^n + dp - mean(dp);  in the cost window, the
//               cell-centred velocity enters a running Welford mean/M2 (Eq. kinenergy) and the four
//               sensors of Sec. 4.1 are sampled (Eq. specific_cost_function).
//
// Boundary rules inside the stencils: a face with one fluid neighbour cell is a wall (normal
// velocity 0, stored as 0); a face with no fluid neighbour takes the mirror value of the
// fluid-side face (no slip by odd reflection; free slip by even reflection on the slip segments of
// the lower wall); free slip at the top, no slip at the bottom, v = 0 at the inlet by reflection
// and dv/dx = 0 at the outlet.
#include "envar_internal.cuh"
#include "../../include/envar.h"

#include <atomic>

namespace envar {

static std::atomic<long long> g_launches{0};
static thread_local bool g_capturing = false;
static thread_local long long g_captured = 0;      // launches recorded into graphs (this thread)
static thread_local bool g_capture_failed = false;
void count_launches(long long n)
{
    if (!g_capturing) g_launches += n;
    else g_captured += n;
}
long long launches_so_far() { return g_launches.load(); }
void set_capturing(bool on)
{
    g_capturing = on;
    if (on) g_capture_failed = false;
}
long long captured_launches() { return g_captured; }
void note_capture_failure() { g_capture_failed = true; }
bool capture_failed() { return g_capture_failed; }

// ---------------------------------------------------------------------------- reset
__global__ void k_broadcast(const double *__restrict__ src, double *__restrict__ dst, long long S, int M)
{
    long long n = S * (long long)M;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        dst[t] = src[t % S];
}

void launch_reset(const Grid &g, int M, const double *u0, const double *v0, double *u, double *v, double *p,
                  double *x, void *Ru, void *Rv, size_t tend_bytes, double *wf, double *wd, int want_welford,
                  MemberCtl *ctl, cudaStream_t st)
{
    size_t bytes = sizeof(double) * (size_t)g.S * M;
    k_broadcast<<<1024, 256, 0, st>>>(u0, u, g.S, M);
    k_broadcast<<<1024, 256, 0, st>>>(v0, v, g.S, M);
    count_launches(2);
    cudaMemsetAsync(p, 0, bytes, st);
    cudaMemsetAsync(x, 0, bytes, st);
    cudaMemsetAsync(Ru, 0, tend_bytes, st);
    cudaMemsetAsync(Rv, 0, tend_bytes, st);
    if (want_welford) cudaMemsetAsync(wf, 0, 3 * bytes, st);
    if (want_welford && wd) cudaMemsetAsync(wd, 0, 3 * bytes, st);
    cudaMemsetAsync(ctl, 0, sizeof(MemberCtl) * M, st);
}

__global__ void k_set_gidx(MemberCtl *ctl, int M, int base)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < M) ctl[m].gidx = base + m;
}
void launch_set_gidx(MemberCtl *ctl, int M, int base, cudaStream_t st)
{
    k_set_gidx<<<cdiv(M, 128), 128, 0, st>>>(ctl, M, base);
    count_launches(1);
}

__global__ void k_copy_status(const MemberCtl *ctl, int M, int *status)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < M) status[m] = ctl[m].status;
}
void launch_copy_status(const MemberCtl *ctl, int M, int *status, cudaStream_t st)
{
    k_copy_status<<<cdiv(M, 128), 128, 0, st>>>(ctl, M, status);
    count_launches(1);
}

// ---------------------------------------------------------------------------- outflow
__global__ void k_outflow(Grid g, const double *__restrict__ u, double *__restrict__ ubc, MemberCtl *ctl)
{
    int m = blockIdx.x;
    const double *um = u + (long long)m * g.S;
    double qin = 0.0, qout = 0.0, nout = 0.0;
    for (int j = threadIdx.x; j < g.ny; j += blockDim.x) {
        long long c = (long long)j * g.P;
        if (g.uk[c] == FK_INLET) qin += g.u_in[j] * g.dy;
        if (g.uk[c + g.nx] == FK_OUTLET) {
            double ub = um[c + g.nx], ui = um[c + g.nx - 1];
            double un = ub - g.dt * g.conv_speed * (ub - ui) / g.dx;
            ubc[(long long)m * g.ny + j] = un;
            qout += un * g.dy;
            nout += 1.0;
        } else {
            ubc[(long long)m * g.ny + j] = 0.0;
        }
    }
    qin = block_reduce(qin, false);
    qout = block_reduce(qout, false);
    nout = block_reduce(nout, false);
    double shift = (nout > 0.0) ? (qin - qout) / (nout * g.dy) : 0.0;
    for (int j = threadIdx.x; j < g.ny; j += blockDim.x)
        if (g.uk[(long long)j * g.P + g.nx] == FK_OUTLET) ubc[(long long)m * g.ny + j] += shift;
    if (threadIdx.x == 0) {
        ctl[m].step += 1;
        ctl[m].outer_done = 0;
        ctl[m].inner_done = 0;
    }
}

void launch_outflow(const Grid &g, int M, const double *u, double *ubc, MemberCtl *ctl, cudaStream_t st)
{
    k_outflow<<<M, 256, 0, st>>>(g, u, ubc, ctl);
    count_launches(1);
}

// ---------------------------------------------------------------------------- predictor (K1)
__device__ __forceinline__ double cell_forcing(const Grid &g, const double *__restrict__ fr, int comp, int i, int j)
{
    int a = i - g.ia, b = j - g.ja;
    if (a < 0 || a >= g.nrx || b < 0 || b >= g.nry) return 0.0;
    return fr[((long long)comp * g.nry + b) * g.nrx + a];
}

template <class TR>
__global__ void __launch_bounds__(256) k_predict(Grid g, const double *__restrict__ u, const double *__restrict__ v,
                                                 const double *__restrict__ p, TR *__restrict__ Ru,
                                                 TR *__restrict__ Rv, double *__restrict__ us,
                                                 double *__restrict__ vs, const double *__restrict__ ubc,
                                                 const double *__restrict__ frect, const MemberCtl *__restrict__ ctl)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int m = blockIdx.z;
    if (i > g.nx || j > g.ny) return;
    const long long off = (long long)m * g.S;
    const double *um = u + off, *vm = v + off, *pm = p + off;
    const double *fr = frect + (long long)m * 2 * g.nry * g.nrx;
    const long long c = (long long)j * g.P + i;
    const int P = g.P;
    const bool first = (ctl[m].step == 1);
    const TR c1 = first ? TR(1) : TR(1.5), c0 = first ? TR(0) : TR(-0.5);
    const TR i4dx = TR(0.25 / g.dx), i4dy = TR(0.25 / g.dy);
    const TR nudx2 = TR(g.nu / (g.dx * g.dx)), nudy2 = TR(g.nu / (g.dy * g.dy));
    const double dt = g.dt;

    if (j < g.ny) {  // u face (i, j)
        uint8_t k = g.uk[c];
        double out;
        if (k == FK_UNK) {
            TR uc = (TR)um[c], ue = (TR)um[c + 1], uw = (TR)um[c - 1];
            const uint8_t kn = (j + 1 < g.ny) ? g.uk[c + P] : FK_ZERO, ks = (j > 0) ? g.uk[c - P] : FK_ZERO;
            TR un = (j + 1 == g.ny) ? uc : (kn == FK_SOLID ? -uc : (kn == FK_SLIP ? uc : (TR)um[c + P]));
            TR usv = (j == 0) ? -uc : (ks == FK_SOLID ? -uc : (ks == FK_SLIP ? uc : (TR)um[c - P]));
            TR vnw = (TR)vm[c + P - 1], vne = (TR)vm[c + P], vsw = (TR)vm[c - 1], vse = (TR)vm[c];
            TR fe = uc + ue, fw = uw + uc;
            TR adv = (fe * fe - fw * fw) * i4dx + ((uc + un) * (vnw + vne) - (usv + uc) * (vsw + vse)) * i4dy;
            TR dif = nudx2 * (ue - TR(2) * uc + uw) + nudy2 * (un - TR(2) * uc + usv);
            TR R = dif - adv;
            TR Rp = Ru[off + c];
            Ru[off + c] = R;
            double f = 0.5 * (cell_forcing(g, fr, 0, i - 1, j) + cell_forcing(g, fr, 0, i, j));
            out = um[c] + dt * (double)(c1 * R + c0 * Rp) + dt * f - dt * (pm[c] - pm[c - 1]) / g.dx;
        } else if (k == FK_INLET) {
            out = g.u_in[j];
        } else if (k == FK_OUTLET) {
            out = ubc[(long long)m * g.ny + j];
        } else {
            out = 0.0;
        }
        us[off + c] = out;
    }
    if (i < g.nx) {  // v face (i, j)
        uint8_t k = g.vk[c];
        double out = 0.0;
        if (k == FK_UNK) {
            TR vc = (TR)vm[c], vn = (TR)vm[c + P], vsv = (TR)vm[c - P];
            TR ve = (i + 1 == g.nx) ? vc : (g.vk[c + 1] == FK_SOLID ? -vc : (TR)vm[c + 1]);
            TR vw = (i == 0) ? -vc : (g.vk[c - 1] == FK_SOLID ? -vc : (TR)vm[c - 1]);
            TR use = (TR)um[c - P + 1], une = (TR)um[c + 1], usw = (TR)um[c - P], unw = (TR)um[c];
            TR fn = vc + vn, fs = vsv + vc;
            TR adv = ((use + une) * (vc + ve) - (usw + unw) * (vw + vc)) * i4dx + (fn * fn - fs * fs) * i4dy;
            TR dif = nudx2 * (ve - TR(2) * vc + vw) + nudy2 * (vn - TR(2) * vc + vsv);
            TR R = dif - adv;
            TR Rp = Rv[off + c];
            Rv[off + c] = R;
            double f = 0.5 * (cell_forcing(g, fr, 1, i, j - 1) + cell_forcing(g, fr, 1, i, j));
            out = vm[c] + dt * (double)(c1 * R + c0 * Rp) + dt * f - dt * (pm[c] - pm[c - P]) / g.dy;
        }
        vs[off + c] = out;
    }
}

template <class TR>
void launch_predict(const Grid &g, int M, const double *u, const double *v, const double *p, TR *Ru, TR *Rv,
                    double *us, double *vs, const double *ubc, const double *frect, const MemberCtl *ctl,
                    cudaStream_t st)
{
    dim3 blk(32, 8), grd(cdiv(g.nx + 1, 32), cdiv(g.ny + 1, 8), M);
    k_predict<TR><<<grd, blk, 0, st>>>(g, u, v, p, Ru, Rv, us, vs, ubc, frect, ctl);
    count_launches(1);
}
template void launch_predict<float>(const Grid &, int, const double *, const double *, const double *, float *,
                                    float *, double *, double *, const double *, const double *,
                                    const MemberCtl *, cudaStream_t);
template void launch_predict<double>(const Grid &, int, const double *, const double *, const double *, double *,
                                     double *, double *, double *, const double *, const double *,
                                     const MemberCtl *, cudaStream_t);

// ---------------------------------------------------------------------------- rhs
__global__ void k_rhs(Grid g, const double *__restrict__ us, const double *__restrict__ vs, double *__restrict__ b)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int m = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const long long off = (long long)m * g.S, c = (long long)j * g.P + i;
    double r = 0.0;
    if (g.fluid[c]) {
        double du = us[off + c + 1] - us[off + c];
        double dv = vs[off + c + g.P] - vs[off + c];
        r = -(g.dy * du + g.dx * dv) / g.dt;
    }
    b[off + c] = r;
}

void launch_rhs(const Grid &g, int M, const double *us, const double *vs, double *b, MemberCtl *, cudaStream_t st)
{
    dim3 blk(32, 8), grd(cdiv(g.nx, 32), cdiv(g.ny, 8), M);
    k_rhs<<<grd, blk, 0, st>>>(g, us, vs, b);
    count_launches(1);
}

// ---------------------------------------------------------------------------- correction (K6)
// Corrected (n+1) velocity of u face c from the predictor and the pressure increment.
__device__ __forceinline__ double u_new(const Grid &g, const double *us, const double *x, long long c)
{
    return (g.uk[c] == FK_UNK) ? us[c] - g.dt * (x[c] - x[c - 1]) / g.dx : us[c];
}
__device__ __forceinline__ double v_new(const Grid &g, const double *vs, const double *x, long long c)
{
    return (g.vk[c] == FK_UNK) ? vs[c] - g.dt * (x[c] - x[c - g.P]) / g.dy : vs[c];
}

// Bilinear sensor samples at (0.2 q, 0), q = 1..4, of the corrected velocity.
__device__ void sample_sensors(const Grid &g, double x0, double y0, const double *us, const double *vs,
                               const double *x, double *out)
{
    for (int q = 0; q < 4; ++q) {
        double xs = 0.2 * (q + 1), ys = 0.0;
        {   // u: faces at (x0 + i dx, y0 + (j + 1/2) dy)
            double fi = (xs - x0) / g.dx, fj = (ys - y0) / g.dy - 0.5;
            int i0 = (int)floor(fi), j0 = (int)floor(fj);
            if (i0 < 0 || i0 + 1 > g.nx || j0 < 0 || j0 + 1 > g.ny - 1) {
                out[2 * q] = nan("");
            } else {
                double tx = fi - i0, ty = fj - j0;
                long long c00 = (long long)j0 * g.P + i0;
                double a = (1 - tx) * u_new(g, us, x, c00) + tx * u_new(g, us, x, c00 + 1);
                double b = (1 - tx) * u_new(g, us, x, c00 + g.P) + tx * u_new(g, us, x, c00 + g.P + 1);
                out[2 * q] = (1 - ty) * a + ty * b;
            }
        }
        {   // v: faces at (x0 + (i + 1/2) dx, y0 + j dy)
            double fi = (xs - x0) / g.dx - 0.5, fj = (ys - y0) / g.dy;
            int i0 = (int)floor(fi), j0 = (int)floor(fj);
            if (i0 < 0 || i0 + 1 > g.nx - 1 || j0 < 0 || j0 + 1 > g.ny) {
                out[2 * q + 1] = nan("");
            } else {
                double tx = fi - i0, ty = fj - j0;
                long long c00 = (long long)j0 * g.P + i0;
                double a = (1 - tx) * v_new(g, vs, x, c00) + tx * v_new(g, vs, x, c00 + 1);
                double b = (ty > 0.0) ? (1 - tx) * v_new(g, vs, x, c00 + g.P) + tx * v_new(g, vs, x, c00 + g.P + 1)
                                      : 0.0;
                out[2 * q + 1] = (1 - ty) * a + ty * b;
            }
        }
    }
}

// Welford step of the window sample n (1-based) of a two-component quantity (a, b) into its
// running means and summed squared deviation M2 (Welford 1962, with a shared count).
__device__ __forceinline__ void welford2(double a, double b, int n, double *ma, double *mb, double *m2)
{
    const double inv_n = 1.0 / (double)n;
    const double da = a - *ma, db = b - *mb;
    const double na = *ma + da * inv_n, nb = *mb + db * inv_n;
    *m2 += da * (a - na) + db * (b - nb);
    *ma = na;
    *mb = nb;
}

__global__ void __launch_bounds__(256) k_correct(Grid g, double x0, double y0, double *__restrict__ u,
                                                 double *__restrict__ v, double *__restrict__ p,
                                                 const double *__restrict__ us, const double *__restrict__ vs,
                                                 const double *__restrict__ x, double *__restrict__ wf,
                                                 double *__restrict__ wd, RefMember ref, int want_welford,
                                                 double *__restrict__ series, Partials pt, MemberCtl *ctl,
                                                 double div_tol, long long nfluid)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int m = blockIdx.z;
    const long long off = (long long)m * g.S;
    const long long c = (long long)j * g.P + i;
    const double *usm = us + off, *vsm = vs + off, *xm = x + off;
    __shared__ double s_mean;
    __shared__ int s_t, s_gm;
    int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if (tid == 0) {
        s_mean = pt.red[m].val[RS_XSUM] / (double)nfluid;
        s_t = ctl[m].step - (g.n_steps - g.n_window);
        s_gm = ctl[m].gidx;
    }
    __syncthreads();
    const double xmean = s_mean;
    const int t = (s_t > 0 && s_t <= g.n_window) ? s_t : 0;  // window sample index (1-based), 0 outside
    const int gm = s_gm;
    int bad = 0;
    if (i <= g.nx && j <= g.ny) {
        if (j < g.ny) {
            double un = u_new(g, usm, xm, c);
            u[off + c] = un;
            bad |= !isfinite(un) ? ENVAR_ST_NONFINITE : 0;
            bad |= (fabs(un) * g.dt > g.dx) ? ENVAR_ST_CFL : 0;
        }
        if (i < g.nx) {
            double vn = v_new(g, vsm, xm, c);
            v[off + c] = vn;
            bad |= !isfinite(vn) ? ENVAR_ST_NONFINITE : 0;
            bad |= (fabs(vn) * g.dt > g.dy) ? ENVAR_ST_CFL : 0;
        }
        if (i < g.nx && j < g.ny && g.fluid[c]) {
            p[off + c] += xm[c] - xmean;
            if (want_welford && t > 0) {
                double uc = 0.5 * (u_new(g, usm, xm, c) + u_new(g, usm, xm, c + 1));
                double vc = 0.5 * (v_new(g, vsm, xm, c) + v_new(g, vsm, xm, c + g.P));
                double *mu = wf + 3 * off, *mv = mu + g.S, *m2 = mv + g.S;
                welford2(uc, vc, t, mu + c, mv + c, m2 + c);
                // d = u - u_0 (Eq. fdapprox times eps, before the window mean is removed)
                double u0c = 0.0, v0c = 0.0;
                bool have0 = false;
                if (ref.traj) {
                    double *tr = ref.traj + (long long)(t - 1) * 2 * g.S;
                    if (gm == 0) { tr[c] = uc; tr[g.S + c] = vc; }
                    else { u0c = tr[c]; v0c = tr[g.S + c]; have0 = true; }
                } else if (ref.us && gm != 0) {
                    u0c = 0.5 * (u_new(g, ref.us, ref.x, c) + u_new(g, ref.us, ref.x, c + 1));
                    v0c = 0.5 * (v_new(g, ref.vs, ref.x, c) + v_new(g, ref.vs, ref.x, c + g.P));
                    have0 = true;
                }
                if (have0 && wd) {
                    double *da = wd + 3 * off, *db = da + g.S, *d2 = db + g.S;
                    welford2(uc - u0c, vc - v0c, t, da + c, db + c, d2 + c);
                }
            }
        }
    }
    bad = __syncthreads_or(bad);
    if (tid == 0 && bad) atomicOr(&ctl[m].status, bad);
    if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
        double dv = g.dt * pt.red[m].val[RS_RMAX] / g.hxy;
        if (dv > ctl[m].max_div) ctl[m].max_div = dv;
        if (!(dv <= div_tol)) ctl[m].status |= ENVAR_ST_DIVERGENCE;
        if (t > 0 && series) {
            double s[8];
            sample_sensors(g, x0, y0, usm, vsm, xm, s);
            double *dst = series + ((long long)m * g.n_window + (t - 1)) * 8;
            for (int q = 0; q < 8; ++q) dst[q] = s[q];
        }
    }
}

void launch_correct(const Grid &g, double x0, double y0, int M, double *u, double *v, double *p,
                    const double *us, const double *vs, const double *x, double *wf, double *wd, RefMember ref,
                    int want_welford, double *series, const Partials &pt, MemberCtl *ctl, double div_tol,
                    long long nfluid, cudaStream_t st)
{
    dim3 blk(32, 8), grd(cdiv(g.nx + 1, 32), cdiv(g.ny + 1, 8), M);
    k_correct<<<grd, blk, 0, st>>>(g, x0, y0, u, v, p, us, vs, x, wf, wd, ref, want_welford, series, pt, ctl,
                                   div_tol, nfluid);
    count_launches(1);
}

// The increment dp is also the next step's initial guess.  The Neumann problem fixes it only up
// to a constant, which the solves leave to drift; a large constant costs accuracy in A x (rounding
// scales with |x|), so the guess is re-centred on the fluid mean once the step has used it.
__global__ void k_recenter(Grid g, double *__restrict__ x, Partials pt, long long nfluid)
{
    const int m = blockIdx.z;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const long long c = (long long)j * g.P + i;
    if (g.fluid[c]) x[(long long)m * g.S + c] -= pt.red[m].val[RS_XSUM] / (double)nfluid;
}

void launch_recenter(const Grid &g, int M, double *x, const Partials &pt, long long nfluid, cudaStream_t st)
{
    dim3 blk(32, 8), grd(cdiv(g.nx, 32), cdiv(g.ny, 8), M);
    k_recenter<<<grd, blk, 0, st>>>(g, x, pt, nfluid);
    count_launches(1);
}

// ---------------------------------------------------------------------------- costs (K7)
// Per-member partial sums over fluid cells of one plane (member stride mstride).
__global__ void k_plane_partial(Grid g, const double *__restrict__ plane, long long mstride, double *__restrict__ part)
{
    int m = blockIdx.y;
    const double *a = plane + (long long)m * mstride;
    long long ncell = (long long)g.ny * g.P;
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x) {
        int i = (int)(c % g.P);
        if (i < g.nx && g.fluid[c]) acc += a[c];
    }
    acc = block_reduce(acc, false);
    if (threadIdx.x == 0) part[(long long)m * gridDim.x + blockIdx.x] = acc;
}

__global__ void k_cost_final(Grid g, const double *__restrict__ part, const double *__restrict__ part_d, int nparts,
                             const double *__restrict__ series, double *__restrict__ Jd, double *__restrict__ Js,
                             double *__restrict__ Yd)
{
    int m = blockIdx.x;
    double acc = 0.0, accd = 0.0;
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) {
        if (part) acc += part[(long long)m * nparts + k];
        if (part_d) accd += part_d[(long long)m * nparts + k];
    }
    acc = block_reduce(acc, false);
    accd = block_reduce(accd, false);
    // sensors: two-pass over the window series
    double js = 0.0;
    int nw = g.n_window;
    if (series && nw > 0) {
        const double *s = series + (long long)m * nw * 8;
        for (int q = 0; q < 8; ++q) {
            double sm = 0.0;
            for (int t = threadIdx.x; t < nw; t += blockDim.x) sm += s[(long long)t * 8 + q];
            sm = block_reduce(sm, false) / nw;
            double sq = 0.0;
            for (int t = threadIdx.x; t < nw; t += blockDim.x) {
                double d = s[(long long)t * 8 + q] - sm;
                sq += d * d;
            }
            js += block_reduce(sq, false);
        }
    }
    if (threadIdx.x == 0) {
        Jd[m] = (nw > 0) ? acc * g.hxy / (2.0 * nw) : 0.0;
        Js[m] = 0.5 * js;
        if (Yd) Yd[m] = (nw > 0) ? accd * g.hxy / (2.0 * nw) : 0.0;
    }
}

void launch_cost_final(const Grid &g, int M, const double *part, const double *part_d, int nparts,
                       const double *series, double *J_domain, double *J_sensor, double *Yd, cudaStream_t st)
{
    k_cost_final<<<M, 256, 0, st>>>(g, part, part_d, nparts, series, J_domain, J_sensor, Yd);
    count_launches(1);
}

void launch_cost(const Grid &g, int M, const double *wf, const double *wd, const double *series, double *J_domain,
                 double *J_sensor, double *Yd, double *part, cudaStream_t st)
{
    const int nparts = 64;
    double *part_d = part + (long long)nparts * M;
    if (wf) {
        dim3 grd(nparts, M);
        k_plane_partial<<<grd, 256, 0, st>>>(g, wf + 2 * g.S, 3 * g.S, part);
        count_launches(1);
    }
    if (wd) {
        dim3 grd(nparts, M);
        k_plane_partial<<<grd, 256, 0, st>>>(g, wd + 2 * g.S, 3 * g.S, part_d);
        count_launches(1);
    }
    launch_cost_final(g, M, wf ? part : nullptr, wd ? part_d : nullptr, nparts, series, J_domain, J_sensor,
                      wd ? Yd : nullptr, st);
}

// ---------------------------------------------------------------------------- state export
__global__ void k_export(Grid g, const double *__restrict__ u, const double *__restrict__ v,
                         const double *__restrict__ p, double *uo, double *vo, double *po)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > g.nx || j > g.ny) return;
    long long c = (long long)j * g.P + i;
    if (uo && j < g.ny) uo[(long long)j * (g.nx + 1) + i] = u[c];
    if (vo && i < g.nx) vo[(long long)j * g.nx + i] = v[c];
    if (po && i < g.nx && j < g.ny) po[(long long)j * g.nx + i] = g.fluid[c] ? p[c] : 0.0;
}

void launch_export_state(const Grid &g, const double *u, const double *v, const double *p, double *uo, double *vo,
                         double *po, cudaStream_t st)
{
    dim3 blk(32, 8), grd(cdiv(g.nx + 1, 32), cdiv(g.ny + 1, 8), 1);
    k_export<<<grd, blk, 0, st>>>(g, u, v, p, uo, vo, po);
    count_launches(1);
}

// Load raw initial fields (compact layouts) into the padded layout, applying the face rules.
__global__ void k_load_ic(Grid g, const double *__restrict__ u0, const double *__restrict__ v0, double *u, double *v)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > g.nx || j > g.ny) return;
    long long c = (long long)j * g.P + i;
    if (j < g.ny) {
        uint8_t k = g.uk[c];
        double val = 0.0;
        if (k == FK_UNK || k == FK_OUTLET) val = u0[(long long)j * (g.nx + 1) + i];
        else if (k == FK_INLET) val = g.u_in[j];
        u[c] = val;
    }
    if (i < g.nx) v[c] = (g.vk[c] == FK_UNK) ? v0[(long long)j * g.nx + i] : 0.0;
}

void launch_load_ic(const Grid &g, const double *u0, const double *v0, double *u, double *v, cudaStream_t st)
{
    dim3 blk(32, 8), grd(cdiv(g.nx + 1, 32), cdiv(g.ny + 1, 8), 1);
    k_load_ic<<<grd, blk, 0, st>>>(g, u0, v0, u, v);
    count_launches(1);
}

} // namespace envar
