// k_mixed.cu -- mixed-precision time step (ENVAR_MIXED) of the forced Navier-Stokes solver.
//
// Same discretisation as k_flow.cu (Sec. 2, Eq. forced_NS on the MAC grid; AB2 + incremental
// projection), with the precision split chosen for GB300, whose FP64 pipe runs at ~1/64 of FP32:
//   * tendencies R (advection, diffusion) in FP32 from the high words of the velocity;
//   * velocity state u, v, the Poisson right-hand side b and solution x, and the Welford
//     accumulators in double-float (hi + lo floats, ~48 bits, df64.cuh), so that the FP64-level
//     divergence tolerance (1e-10) is met without FP64 instructions per cell;
//   * pressure p in FP32: u^{n+1} = P(u^n + dt R) does not depend on the accuracy of p^n, which
//     only shifts the incremental solve's starting point.
// The projection operators are built from df64 constants with dt*c = h*gamma, so the divergence
// of the corrected field equals -dt (b - A x)/(dx dy) to df64 rounding.
#include "df64.cuh"
#include "envar_internal.cuh"
#include "res_finish.cuh"
#include "../../include/envar.h"

namespace envar {

// ---------------------------------------------------------------------------- IC / reset / export
__global__ void k_load_ic_mx(Grid g, const double *__restrict__ u0, const double *__restrict__ v0, float *uh, float *ul,
                             float *vh, float *vl)
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
        f2 d = d_to_df(val);
        uh[c] = d.h; ul[c] = d.l;
    }
    if (i < g.nx) {
        f2 d = d_to_df((g.vk[c] == FK_UNK) ? v0[(long long)j * g.nx + i] : 0.0);
        vh[c] = d.h; vl[c] = d.l;
    }
}

void launch_load_ic_mx(const Grid &g, const double *u0, const double *v0, const MixState &s0, cudaStream_t st)
{
    dim3 blk(32, 8), grd(cdiv(g.nx + 1, 32), cdiv(g.ny + 1, 8), 1);
    k_load_ic_mx<<<grd, blk, 0, st>>>(g, u0, v0, s0.uh, s0.ul, s0.vh, s0.vl);
    count_launches(1);
}

__global__ void k_broadcast4(const float *__restrict__ a, const float *__restrict__ b, const float *__restrict__ c,
                             const float *__restrict__ d, float *A, float *B, float *C, float *D, long long S, int M)
{
    long long n = S * (long long)M;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        long long k = t % S;
        A[t] = a[k]; B[t] = b[k]; C[t] = c[k]; D[t] = d[k];
    }
}

void launch_reset_mx(const Grid &g, int M, const MixState &ic, const MixState &s, MemberCtl *ctl, int want_welford,
                     cudaStream_t st)
{
    size_t fb = sizeof(float) * (size_t)g.S * M;
    k_broadcast4<<<1024, 256, 0, st>>>(ic.uh, ic.ul, ic.vh, ic.vl, s.uh, s.ul, s.vh, s.vl, g.S, M);
    count_launches(1);
    cudaMemsetAsync(s.p, 0, fb, st);
    cudaMemsetAsync(s.xh, 0, fb, st);
    cudaMemsetAsync(s.xl, 0, fb, st);
    cudaMemsetAsync(s.Ru, 0, fb, st);
    cudaMemsetAsync(s.Rv, 0, fb, st);
    cudaMemsetAsync(s.Ru + s.rstride, 0, fb, st);
    cudaMemsetAsync(s.Rv + s.rstride, 0, fb, st);
    if (want_welford) cudaMemsetAsync(s.wf, 0, 6 * fb, st);
    if (want_welford && s.wd) cudaMemsetAsync(s.wd, 0, 4 * fb, st);
    cudaMemsetAsync(ctl, 0, sizeof(MemberCtl) * M, st);
}

__global__ void k_export_mx(Grid g, const float *uh, const float *ul, const float *vh, const float *vl, const float *p,
                            double *uo, double *vo, double *po)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > g.nx || j > g.ny) return;
    long long c = (long long)j * g.P + i;
    if (uo && j < g.ny) uo[(long long)j * (g.nx + 1) + i] = (double)uh[c] + (double)ul[c];
    if (vo && i < g.nx) vo[(long long)j * g.nx + i] = (double)vh[c] + (double)vl[c];
    if (po && i < g.nx && j < g.ny) po[(long long)j * g.nx + i] = g.fluid[c] ? (double)p[c] : 0.0;
}

void launch_export_mx(const Grid &g, const MixState &s, long long off, double *uo, double *vo, double *po,
                      cudaStream_t st)
{
    dim3 blk(32, 8), grd(cdiv(g.nx + 1, 32), cdiv(g.ny + 1, 8), 1);
    k_export_mx<<<grd, blk, 0, st>>>(g, s.uh + off, s.ul + off, s.vh + off, s.vl + off, s.p + off, uo, vo, po);
    count_launches(1);
}

// ---------------------------------------------------------------------------- outflow
__global__ void k_outflow_mx(Grid g, const float *__restrict__ uh, const float *__restrict__ ul, double *__restrict__ ubc,
                             MemberCtl *ctl)
{
    int m = blockIdx.x;
    const long long off = (long long)m * g.S;
    double qin = 0.0, qout = 0.0, nout = 0.0;
    for (int j = threadIdx.x; j < g.ny; j += blockDim.x) {
        long long c = (long long)j * g.P;
        if (g.uk[c] == FK_INLET) qin += g.u_in[j] * g.dy;
        if (g.uk[c + g.nx] == FK_OUTLET) {
            double ub = (double)uh[off + c + g.nx] + (double)ul[off + c + g.nx];
            double ui = (double)uh[off + c + g.nx - 1] + (double)ul[off + c + g.nx - 1];
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

void launch_outflow_mx(const Grid &g, int M, const MixState &s, double *ubc, MemberCtl *ctl, cudaStream_t st)
{
    k_outflow_mx<<<M, 256, 0, st>>>(g, s.uh, s.ul, ubc, ctl);
    count_launches(1);
}

// ---------------------------------------------------------------------------- predictor (K1)
__device__ __forceinline__ float cell_forcing_f(const Grid &g, const float *__restrict__ fr, int comp, int i, int j)
{
    int a = i - g.ia, b = j - g.ja;
    if (a < 0 || a >= g.nrx || b < 0 || b >= g.nry) return 0.f;
    return fr[((long long)comp * g.nry + b) * g.nrx + a];
}

// Tendencies are double-buffered by step parity (s.Ru / s.Ru + s.rstride, likewise Rv): a block
// also computes the predictor on the first face column and row of its east and north neighbours
// (their Poisson right-hand side needs it) and must read the previous step's tendency there while
// the neighbouring block writes the new one.
struct RBuf { const float *uin, *vin; float *uout, *vout; };
__device__ __forceinline__ RBuf rbuf(const MixState &s, long long off, int step)
{
    const long long a = (step & 1) ? 0 : s.rstride, b = (step & 1) ? s.rstride : 0;
    return RBuf{s.Ru + off + a, s.Rv + off + a, s.Ru + off + b, s.Rv + off + b};
}

// Predictor on u face (i, j) of member m: R = diffusion - advection (central, divergence form, FP32 on
// the high words), u* = u^n + dt (c1 R + c0 R^{n-1}) - dt G p^n + dt f on an unknown face (df64 sum),
// the inlet profile or the convective outlet value on boundary faces, 0 on walls.  Rout (nullable)
// receives R.  The owner of a face and the neighbouring block that recomputes it must get the same
// bits (a last-bit difference between the stored u* and the u* of the right-hand side leaves a
// divergence the pressure solve cannot remove), so every FP32 operation is an explicitly rounded
// intrinsic, which the compiler may not contract into an FMA differently at the two call sites.
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }

__device__ __forceinline__ f2 ustar_mx(const Grid &g, const MixConst &K, const MixState &s, long long off, int m, int i,
                                       int j, const float *__restrict__ Rin, float *Rout, const double *__restrict__ ubc,
                                       const float *__restrict__ inh, const float *__restrict__ inl, float c1, float c0)
{
    const int P = g.P;
    const long long c = (long long)j * P + i;
    const uint8_t ku = g.uk[c];
    if (ku == FK_INLET) return f2{inh[j], inl[j]};
    if (ku == FK_OUTLET) return d_to_df(ubc[(long long)m * g.ny + j]);
    if (ku != FK_UNK) return f2{0.f, 0.f};
    const float *__restrict__ uh = s.uh + off;
    const float *__restrict__ vh = s.vh + off;
    const float *__restrict__ pm = s.p + off;
    const int jn = min(j + 1, g.ny - 1), js = max(j - 1, 0), ie = min(i + 1, g.nx), iw = max(i - 1, 0);
    const int jvn = min(j + 1, g.ny);
    const uint8_t kuN = g.uk[(long long)jn * P + i], kuS = g.uk[(long long)js * P + i];
    const float uc = uh[c], ue = uh[(long long)j * P + ie], uw = uh[(long long)j * P + iw];
    const float un0 = uh[(long long)jn * P + i], us0 = uh[(long long)js * P + i];
    const float vc = vh[c], vn = vh[(long long)jvn * P + i], vnw = vh[(long long)jvn * P + iw];
    const float vsw = vh[(long long)j * P + iw];
    const float un = (j + 1 == g.ny) ? uc : (kuN == FK_SOLID ? -uc : (kuN == FK_SLIP ? uc : un0));
    const float usv = (j == 0) ? -uc : (kuS == FK_SOLID ? -uc : (kuS == FK_SLIP ? uc : us0));
    const float fe = fa(uc, ue), fw = fa(uw, uc);
    const float adv = fa(fm(fs(fm(fe, fe), fm(fw, fw)), K.i4dx),
                         fm(fs(fm(fa(uc, un), fa(vnw, vn)), fm(fa(usv, uc), fa(vsw, vc))), K.i4dy));
    const float uc2 = fm(2.f, uc);
    const float dif = fa(fm(K.nudx2, fa(fs(ue, uc2), uw)), fm(K.nudy2, fa(fs(un, uc2), usv)));
    const float R = fs(dif, adv);
    if (Rout) Rout[c] = R;
    const float du = fs(fm(K.dt, fa(fm(c1, R), fm(c0, Rin[c]))), fm(K.gxf, fs(pm[c], pm[(long long)j * P + iw])));
    f2 out = df_add_f(f2{uc, s.ul[off + c]}, du);
    const float *__restrict__ fr = s.frect + (long long)m * 2 * g.nry * g.nrx;
    const float f = fm(0.5f, fa(cell_forcing_f(g, fr, 0, i - 1, j), cell_forcing_f(g, fr, 0, i, j)));
    if (f != 0.f) out = df_add_f(out, fm(K.dt, f));
    return out;
}

// Predictor on v face (i, j) of member m (as ustar_mx; v = 0 on every face but the unknown ones).
__device__ __forceinline__ f2 vstar_mx(const Grid &g, const MixConst &K, const MixState &s, long long off, int m, int i,
                                       int j, const float *__restrict__ Rin, float *Rout, float c1, float c0)
{
    const int P = g.P;
    const long long c = (long long)j * P + i;
    if (g.vk[c] != FK_UNK) return f2{0.f, 0.f};
    const float *__restrict__ uh = s.uh + off;
    const float *__restrict__ vh = s.vh + off;
    const float *__restrict__ pm = s.p + off;
    const int js = max(j - 1, 0), ie = min(i + 1, g.nx);
    const int ivw = max(i - 1, 0), ive = min(i + 1, g.nx - 1), jvn = min(j + 1, g.ny);
    const uint8_t kvE = g.vk[(long long)j * P + ive], kvW = g.vk[(long long)j * P + ivw];
    const float uc = uh[c], ue = uh[(long long)j * P + ie];
    const float use = uh[(long long)js * P + ie], usw = uh[(long long)js * P + i];
    const float vc = vh[c], vn = vh[(long long)jvn * P + i], vs0 = vh[(long long)js * P + i];
    const float ve0 = vh[(long long)j * P + ive], vw0 = vh[(long long)j * P + ivw];
    const float ve = (i + 1 == g.nx) ? vc : (kvE == FK_SOLID ? -vc : ve0);
    const float vw = (i == 0) ? -vc : (kvW == FK_SOLID ? -vc : vw0);
    const float fn = fa(vc, vn), fsf = fa(vs0, vc);
    const float adv = fa(fm(fs(fm(fa(use, ue), fa(vc, ve)), fm(fa(usw, uc), fa(vw, vc))), K.i4dx),
                         fm(fs(fm(fn, fn), fm(fsf, fsf)), K.i4dy));
    const float vc2 = fm(2.f, vc);
    const float dif = fa(fm(K.nudx2, fa(fs(ve, vc2), vw)), fm(K.nudy2, fa(fs(vn, vc2), vs0)));
    const float R = fs(dif, adv);
    if (Rout) Rout[c] = R;
    const float dv = fs(fm(K.dt, fa(fm(c1, R), fm(c0, Rin[c]))), fm(K.gyf, fs(pm[c], pm[(long long)js * P + i])));
    f2 out = df_add_f(f2{vc, s.vl[off + c]}, dv);
    const float *__restrict__ fr = s.frect + (long long)m * 2 * g.nry * g.nrx;
    const float f = fm(0.5f, fa(cell_forcing_f(g, fr, 1, i, j - 1), cell_forcing_f(g, fr, 1, i, j)));
    if (f != 0.f) out = df_add_f(out, fm(K.dt, f));
    return out;
}

// K1: predictor and Poisson right-hand side in one pass.  A 32 x 8 block owns the u and v faces
// (i, j) of its tile and writes u*, v* and the new tendencies; it also computes u* on the tile's
// east face column and v* on its north face row into shared memory, so every cell of the tile has
// the four faces of b = -(dy (u*_E - u*_W) + dx (v*_N - v*_S)) / dt (df64, zero in solid cells)
// on chip; the right-hand side never re-reads u*, v*.
constexpr int PR_TX = 32, PR_TY = 8;
__global__ void __launch_bounds__(PR_TX *PR_TY, 6) k_predict_rhs_mx(Grid g, MixConst K, MixState s,
                                                                const double *__restrict__ ubc,
                                                                const float *__restrict__ inh,
                                                                const float *__restrict__ inl,
                                                                const MemberCtl *__restrict__ ctl,
                                                                const MemberRed *__restrict__ red, float inv_nfluid)
{
    __shared__ float suh[PR_TY][PR_TX + 1], sul[PR_TY][PR_TX + 1];
    __shared__ float svh[PR_TY + 1][PR_TX], svl[PR_TY + 1][PR_TX];
    __shared__ float s_xmean;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = blockIdx.x * PR_TX, j0 = blockIdx.y * PR_TY;
    const int i = i0 + tx, j = j0 + ty;
    const int m = blockIdx.z;
    const long long off = (long long)m * g.S;
    const int step = ctl[m].step;
    const bool first = (step == 1);
    const float c1 = first ? 1.f : 1.5f, c0 = first ? 0.f : -0.5f;
    const RBuf R = rbuf(s, off, step);
    const long long c = (long long)j * g.P + i;
    // the fluid sum of the last increment: loaded by one thread at entry, stored to shared memory
    // after the face updates (its latency overlaps them), read after the barrier
    const bool lead = tx == 0 && ty == 0 && s.xp && step >= 2;
    double xsum = 0.0;
    if (lead) xsum = __ldcg(&red[m].val[RS_XSUM]);
    if (i <= g.nx && j < g.ny) {
        const f2 u = ustar_mx(g, K, s, off, m, i, j, R.uin, R.uout, ubc, inh, inl, c1, c0);
        s.ush[off + c] = u.h; s.usl[off + c] = u.l;
        suh[ty][tx] = u.h; sul[ty][tx] = u.l;
    }
    if (i < g.nx && j <= g.ny) {
        const f2 v = vstar_mx(g, K, s, off, m, i, j, R.vin, R.vout, c1, c0);
        s.vsh[off + c] = v.h; s.vsl[off + c] = v.l;
        svh[ty][tx] = v.h; svl[ty][tx] = v.l;
    }
    // the east face column and north face row belong to the neighbouring tiles: recompute them here
    if (tx == 0) {
        const int ie = i0 + PR_TX;
        if (ie <= g.nx && j < g.ny) {
            const f2 u = ustar_mx(g, K, s, off, m, ie, j, R.uin, nullptr, ubc, inh, inl, c1, c0);
            suh[ty][PR_TX] = u.h; sul[ty][PR_TX] = u.l;
        }
    }
    if (ty == 0) {
        const int jn = j0 + PR_TY;
        if (i < g.nx && jn <= g.ny) {
            const f2 v = vstar_mx(g, K, s, off, m, i, jn, R.vin, nullptr, c1, c0);
            svh[PR_TY][tx] = v.h; svl[PR_TY][tx] = v.l;
        }
    }
    if (lead) s_xmean = (float)xsum * inv_nfluid;
    __syncthreads();
    if (i < g.nx && j < g.ny) {
        f2 b{0.f, 0.f};
        if (g.fluid[c]) {
            // initial guess of this step's pressure increment (no other kernel of the step reads x yet)
            if (s.xp && step >= 2) {
                const f2 xr = df_add_f(f2{s.xh[off + c], s.xl[off + c]}, -s_xmean);
                f2 guess = xr;                                // from the third step: 2 dp^n - dp^(n-1)
                if (step >= 3) guess = df_add_f(f2{2.f * xr.h, 2.f * xr.l}, -s.xp[off + c]);
                s.xp[off + c] = xr.h;
                s.xh[off + c] = guess.h;
                s.xl[off + c] = guess.l;
            }
            const f2 dU = df_sub(f2{suh[ty][tx + 1], sul[ty][tx + 1]}, f2{suh[ty][tx], sul[ty][tx]});
            const f2 dV = df_sub(f2{svh[ty + 1][tx], svl[ty + 1][tx]}, f2{svh[ty][tx], svl[ty][tx]});
            b = df_add(df_mul(dU, f2{K.kxh, K.kxl}), df_mul(dV, f2{K.kyh, K.kyl}));
            b = f2{-b.h, -b.l};
        }
        s.bh[off + c] = b.h;
        s.bl[off + c] = b.l;
    }
}

void launch_predict_rhs_mx(const Grid &g, const MixConst &K, int M, const MixState &s, const double *ubc,
                           const float *inh, const float *inl, const MemberCtl *ctl, const MemberRed *red,
                           long long nfluid, cudaStream_t st)
{
    dim3 blk(PR_TX, PR_TY), grd(cdiv(g.nx + 1, PR_TX), cdiv(g.ny + 1, PR_TY), M);
    k_predict_rhs_mx<<<grd, blk, 0, st>>>(g, K, s, ubc, inh, inl, ctl, red, (float)(1.0 / (double)nfluid));
    count_launches(1);
}

// ---------------------------------------------------------------------------- outer residual (df64)
// k_outer_residual_mx: r = b - A x in df64 on every fluid cell (FP32 r = its leading word; 0 on the
// other cells), e = 0, and per block the maximum |r| and the fluid sum of x as partials (no ticket:
// the totals, the convergence test and the refinement count are formed after the kernel by one
// warp per member, res_finish_member).  A warp owns a
// 64-column strip of OR_ROWS rows, lane l the cell pair (2l, 2l+1): x of the strip's rows and of
// the rows above and below, b, the open-face and fluid bits and the strip's edge cells are all
// loaded first (in flight together, before the control word is tested), east / west neighbours
// come from the neighbouring lanes by shuffle, and the level-0 open-face bits select the
// operator's terms (an open face joins two fluid cells).
constexpr int OR_ROWS = 4, OR_WARPS = 8;

__global__ void __launch_bounds__(OR_WARPS * 32) k_outer_residual_mx(Grid g, Level L0, MixConst K,
                                                                     const float *__restrict__ bh,
                                                                     const float *__restrict__ bl,
                                                                     const float *__restrict__ xh,
                                                                     const float *__restrict__ xl,
                                                                     float *__restrict__ r, float *__restrict__ e,
                                                                     RedCtx rc, const MemberCtl *ctl)
{
    constexpr int R = OR_ROWS, NR = OR_ROWS + 2;
    const int m = blockIdx.z;
    const long long off = (long long)m * g.S;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int iL = blockIdx.x * 64 + 2 * lane;
    const bool colok = iL < g.nx;                               // nx is even: both cells of the pair
    const int j0 = (blockIdx.y * OR_WARPS + w) * OR_ROWS;
    const float *xhm = xh + off, *xlm = xl + off;
    float2 xrh[NR], xrl[NR], brh[R], brl[R];
    f2 xw[R], xe[R];
    unsigned int ob[R], fl[R];
#pragma unroll
    for (int q = 0; q < NR; ++q) {                              // rows j0 - 1 .. j0 + R; zeros outside
        const int j = j0 - 1 + q;
        xrh[q] = xrl[q] = make_float2(0.f, 0.f);
        if (colok && j >= 0 && j < g.ny) {
            const long long c = (long long)j * g.P + iL;
            xrh[q] = ld_early_nc(reinterpret_cast<const float2 *>(xhm + c));
            xrl[q] = ld_early_nc(reinterpret_cast<const float2 *>(xlm + c));
        }
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int j = j0 + q;
        brh[q] = brl[q] = make_float2(0.f, 0.f);
        xw[q] = xe[q] = f2{0.f, 0.f};
        ob[q] = fl[q] = 0u;
        if (j < g.ny) {
            const long long c = (long long)j * g.P + iL;
            if (colok) {
                brh[q] = ld_early_nc(reinterpret_cast<const float2 *>(bh + off + c));
                brl[q] = ld_early_nc(reinterpret_cast<const float2 *>(bl + off + c));
                ob[q] = ld_early_nc_u16(L0.open + c);
                fl[q] = ld_early_nc_u16(g.fluid + c);
            }
            if (lane == 0 && iL >= 1) xw[q] = f2{ld_early_nc(xhm + c - 1), ld_early_nc(xlm + c - 1)};
            if (lane == 31 && iL + 2 < g.nx) xe[q] = f2{ld_early_nc(xhm + c + 2), ld_early_nc(xlm + c + 2)};
        }
    }
    if (ctl[m].outer_done) return;
    const f2 cx{K.cxh, K.cxl}, cy{K.cyh, K.cyl};
    auto cell_r = [&](unsigned int o, f2 xc, f2 xW, f2 xE, f2 xS, f2 xN, f2 b) -> float {
        f2 sx{0.f, 0.f}, sy{0.f, 0.f};
        if (o & 1u) sx = df_add(sx, df_sub(xc, xW));
        if (o & 2u) sx = df_add(sx, df_sub(xc, xE));
        if (o & 4u) sy = df_add(sy, df_sub(xc, xS));
        if (o & 8u) sy = df_add(sy, df_sub(xc, xN));
        const f2 ax = df_add(df_mul(sx, cx), df_mul(sy, cy));
        return df_sub(b, ax).h;
    };
    float rmax = 0.f;
    f2 xs{0.f, 0.f};
    if (j0 < g.ny) {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int j = j0 + q;
            if (j >= g.ny) break;
            const f2 x0{xrh[q + 1].x, xrl[q + 1].x}, x1{xrh[q + 1].y, xrl[q + 1].y};
            f2 xW{__shfl_up_sync(0xffffffffu, x1.h, 1), __shfl_up_sync(0xffffffffu, x1.l, 1)};
            f2 xE{__shfl_down_sync(0xffffffffu, x0.h, 1), __shfl_down_sync(0xffffffffu, x0.l, 1)};
            if (lane == 0) xW = xw[q];
            if (lane == 31) xE = xe[q];
            if (colok) {
                const long long c = (long long)j * g.P + iL;
                float2 rv = make_float2(0.f, 0.f);
                if (fl[q] & 0xffu) {
                    rv.x = cell_r(ob[q] & 15u, x0, xW, x1, f2{xrh[q].x, xrl[q].x}, f2{xrh[q + 2].x, xrl[q + 2].x},
                                  f2{brh[q].x, brl[q].x});
                    rmax = fmaxf(rmax, fabsf(rv.x));
                    xs = df_add_f(xs, x0.h);
                }
                if (fl[q] >> 8) {
                    rv.y = cell_r((ob[q] >> 8) & 15u, x1, x0, xE, f2{xrh[q].y, xrl[q].y}, f2{xrh[q + 2].y, xrl[q + 2].y},
                                  f2{brh[q].y, brl[q].y});
                    rmax = fmaxf(rmax, fabsf(rv.y));
                    xs = df_add_f(xs, x1.h);
                }
                *reinterpret_cast<float2 *>(r + off + c) = rv;
                *reinterpret_cast<float2 *>(e + off + c) = make_float2(0.f, 0.f);
            }
        }
    }
    const float rm = block_max_f(rmax);
    const f2 xsum = block_sum_df(xs);
    if (threadIdx.x == 0) {
        const long long blk = blockIdx.x + gridDim.x * blockIdx.y;
        float *pr = reinterpret_cast<float *>(rc.part + ((long long)RS_RMAX * rc.stride + m) * rc.nblk + blk);
        *pr = rm;
        *reinterpret_cast<float2 *>(rc.part + ((long long)RS_XSUM * rc.stride + m) * rc.nblk + blk) =
            make_float2(xsum.h, xsum.l);
    }
}

__global__ void k_res_finish(RedCtx rc, MemberCtl *ctl, int M, int n, double rtol_abs, int count_it)
{
    if (blockIdx.x < M) res_finish_member(rc, ctl, blockIdx.x, n, rtol_abs, count_it);
}

// k_axpy_last_mx: the last inner CG update fused with the refinement's update of x: e + alpha p is
// formed in registers and added to x in df64 (x += e) on the cells where it is nonzero (the fluid
// cells: e and p vanish elsewhere); r, and e itself, are not needed after the last inner
// iteration.  A member whose inner loop already stopped (inner_done) only takes x += e.  Four
// values per thread (two aligned pairs), pointwise.
__global__ void __launch_bounds__(128) k_axpy_last_mx(Grid g, float *__restrict__ xh, float *__restrict__ xl,
                                                      const float *__restrict__ e, const float *__restrict__ p,
                                                      RedCtx rc, MemberCtl *ctl, int k)
{
    const int m = blockIdx.z;
    const int i = 4 * (blockIdx.x * blockDim.x + threadIdx.x), j = blockIdx.y;
    const long long c = (long long)m * g.S + (long long)j * g.P + i;
    // the data first (none of it depends on the control word or on alpha); pairs past nx are not
    // touched (nx is even: pairs are whole)
    float2 ev[2], pv[2], x0[2], x1[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        ev[h] = pv[h] = x0[h] = x1[h] = make_float2(0.f, 0.f);
        if (i + 2 * h < g.nx) {
            ev[h] = ld_early_nc(reinterpret_cast<const float2 *>(e + c + 2 * h));
            pv[h] = ld_early_nc(reinterpret_cast<const float2 *>(p + c + 2 * h));
            x0[h] = ld_early(reinterpret_cast<const float2 *>(xh + c + 2 * h));
            x1[h] = ld_early(reinterpret_cast<const float2 *>(xl + c + 2 * h));
        }
    }
    if (ctl[m].outer_done) return;
    const bool moving = !ctl[m].inner_done;
    const float a = moving ? rc.red[m].fa : 0.f;   // alpha of this iteration, formed by the SpMV
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (i + 2 * h >= g.nx) break;
        float2 d = ev[h];
        if (moving) {
            d.x += a * pv[h].x;
            d.y += a * pv[h].y;
        }
        if (d.x != 0.f || d.y != 0.f) {
            float2 hi = x0[h], lo = x1[h];
            if (d.x != 0.f) { const f2 sx = df_add_f(f2{hi.x, lo.x}, d.x); hi.x = sx.h; lo.x = sx.l; }
            if (d.y != 0.f) { const f2 sy = df_add_f(f2{hi.y, lo.y}, d.y); hi.y = sy.h; lo.y = sy.l; }
            *reinterpret_cast<float2 *>(xh + c + 2 * h) = hi;
            *reinterpret_cast<float2 *>(xl + c + 2 * h) = lo;
        }
    }
    if (moving && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) ctl[m].inner_its += 1;
}

int outer_residual_parts_mx(const Grid &g) { return cdiv(g.nx, 64) * cdiv(g.ny, OR_WARPS * OR_ROWS); }

void launch_outer_residual_mx(const Grid &g, const Level &L0, const MixConst &K, int M, const MixState &s, float *r,
                              float *e, const RedCtx &rc, MemberCtl *ctl, double rtol_abs, int count_it, int finish,
                              cudaStream_t st)
{
    dim3 grd(cdiv(g.nx, 64), cdiv(g.ny, OR_WARPS * OR_ROWS), M);
    k_outer_residual_mx<<<grd, OR_WARPS * 32, 0, st>>>(g, L0, K, s.bh, s.bl, s.xh, s.xl, r, e, rc, ctl);
    count_launches(1);
    if (finish) {
        k_res_finish<<<M, 32, 0, st>>>(rc, ctl, M, outer_residual_parts_mx(g), rtol_abs, count_it);
        count_launches(1);
    }
}

void launch_axpy_last_mx(const Grid &g, int M, const MixState &s, const float *e, const float *p, const RedCtx &rc,
                         MemberCtl *ctl, int k, cudaStream_t st)
{
    dim3 grd(cdiv(cdiv(g.nx, 4), 128), g.ny, M);
    k_axpy_last_mx<<<grd, 128, 0, st>>>(g, s.xh, s.xl, e, p, rc, ctl, k);
    count_launches(1);
}

// ---------------------------------------------------------------------------- correction (K6)
__device__ __forceinline__ f2 u_new_mx(const Grid &g, const MixConst &K, const float *ush, const float *usl,
                                       const float *xh, const float *xl, long long c)
{
    f2 us{ush[c], usl[c]};
    if (g.uk[c] != FK_UNK) return us;
    f2 d = df_sub(f2{xh[c], xl[c]}, f2{xh[c - 1], xl[c - 1]});
    return df_sub(us, df_mul(d, f2{K.gxh, K.gxl}));
}
__device__ __forceinline__ f2 v_new_mx(const Grid &g, const MixConst &K, const float *vsh, const float *vsl,
                                       const float *xh, const float *xl, long long c)
{
    f2 vs{vsh[c], vsl[c]};
    if (g.vk[c] != FK_UNK) return vs;
    f2 d = df_sub(f2{xh[c], xl[c]}, f2{xh[c - g.P], xl[c - g.P]});
    return df_sub(vs, df_mul(d, f2{K.gyh, K.gyl}));
}

__device__ void sample_sensors_mx(const Grid &g, const MixConst &K, double x0, double y0, const float *ush,
                                  const float *usl, const float *vsh, const float *vsl, const float *xh,
                                  const float *xl, double *out)
{
    for (int q = 0; q < 4; ++q) {
        double xs = 0.2 * (q + 1), ys = 0.0;
        {
            double fi = (xs - x0) / g.dx, fj = (ys - y0) / g.dy - 0.5;
            int i0 = (int)floor(fi), j0 = (int)floor(fj);
            if (i0 < 0 || i0 + 1 > g.nx || j0 < 0 || j0 + 1 > g.ny - 1) {
                out[2 * q] = nan("");
            } else {
                double tx = fi - i0, ty = fj - j0;
                long long c00 = (long long)j0 * g.P + i0;
                double a = (1 - tx) * df_to_d(u_new_mx(g, K, ush, usl, xh, xl, c00)) +
                           tx * df_to_d(u_new_mx(g, K, ush, usl, xh, xl, c00 + 1));
                double b = (1 - tx) * df_to_d(u_new_mx(g, K, ush, usl, xh, xl, c00 + g.P)) +
                           tx * df_to_d(u_new_mx(g, K, ush, usl, xh, xl, c00 + g.P + 1));
                out[2 * q] = (1 - ty) * a + ty * b;
            }
        }
        {
            double fi = (xs - x0) / g.dx - 0.5, fj = (ys - y0) / g.dy;
            int i0 = (int)floor(fi), j0 = (int)floor(fj);
            if (i0 < 0 || i0 + 1 > g.nx - 1 || j0 < 0 || j0 + 1 > g.ny) {
                out[2 * q + 1] = nan("");
            } else {
                double tx = fi - i0, ty = fj - j0;
                long long c00 = (long long)j0 * g.P + i0;
                double a = (1 - tx) * df_to_d(v_new_mx(g, K, vsh, vsl, xh, xl, c00)) +
                           tx * df_to_d(v_new_mx(g, K, vsh, vsl, xh, xl, c00 + 1));
                double b = (ty > 0.0) ? (1 - tx) * df_to_d(v_new_mx(g, K, vsh, vsl, xh, xl, c00 + g.P)) +
                                            tx * df_to_d(v_new_mx(g, K, vsh, vsl, xh, xl, c00 + g.P + 1))
                                      : 0.0;
                out[2 * q + 1] = (1 - ty) * a + ty * b;
            }
        }
    }
}

__device__ __forceinline__ f2 corrected(bool unk, f2 us, f2 xa, f2 xb, f2 gam)
{
    return unk ? df_sub(us, df_mul(df_sub(xa, xb), gam)) : us;
}

// df64 Welford step of the window sample n (1-based) of (a, b) into running means and M2.
__device__ __forceinline__ void welford2_df(f2 a, f2 b, int n, float *w, long long S, long long c)
{
    const f2 inv_n = df_recip_int(n);
    const f2 mu{w[c], w[S + c]}, mv{w[2 * S + c], w[3 * S + c]};
    f2 m2{w[4 * S + c], w[5 * S + c]};
    const f2 du = df_sub(a, mu);
    const f2 mun = df_add(mu, df_mul(du, inv_n));
    const f2 dv = df_sub(b, mv);
    const f2 mvn = df_add(mv, df_mul(dv, inv_n));
    m2 = df_add(m2, df_add(df_mul(du, df_sub(a, mun)), df_mul(dv, df_sub(b, mvn))));
    w[c] = mun.h; w[S + c] = mun.l;
    w[2 * S + c] = mvn.h; w[3 * S + c] = mvn.l;
    w[4 * S + c] = m2.h; w[5 * S + c] = m2.l;
}

// Welford step of the member-minus-member-0 difference d = (a, b), a quantity of the size of the
// perturbation response: FP32 running means, df64 M2 (planes: mean_a, mean_b, M2 hi, M2 lo).
__device__ __forceinline__ void welford2_diff(float a, float b, int n, float *w, long long S, long long c)
{
    const float inv_n = 1.0f / (float)n;
    const float ma = w[c], mb = w[S + c];
    const float da = a - ma, db = b - mb;
    const float na = ma + da * inv_n, nb = mb + db * inv_n;
    f2 m2{w[2 * S + c], w[3 * S + c]};
    m2 = df_add(m2, df_add(two_prod(da, a - na), two_prod(db, b - nb)));
    w[c] = na; w[S + c] = nb;
    w[2 * S + c] = m2.h; w[3 * S + c] = m2.l;
}

__global__ void __launch_bounds__(256, 5) k_correct_mx(Grid g, MixConst K, MixState s, MixState ref, double x0, double y0,
                                                    int want_welford, double *__restrict__ series, Partials pt,
                                                    MemberCtl *ctl, double div_tol, long long nfluid)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int m = blockIdx.z;
    const long long off = (long long)m * g.S;
    const int P = g.P;
    const float *__restrict__ ush = s.ush + off;
    const float *__restrict__ usl = s.usl + off;
    const float *__restrict__ vsh = s.vsh + off;
    const float *__restrict__ vsl = s.vsl + off;
    const float *__restrict__ xh = s.xh + off;
    const float *__restrict__ xl = s.xl + off;
    __shared__ float s_mean;
    __shared__ int s_t, s_gm;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if (tid == 0) {
        s_mean = (float)(pt.red[m].val[RS_XSUM] / (double)nfluid);
        s_t = ctl[m].step - (g.n_steps - g.n_window);
        s_gm = ctl[m].gidx;
    }
    __syncthreads();
    const float xmean = s_mean;
    const int t = (s_t > 0 && s_t <= g.n_window) ? s_t : 0;
    const int gm = s_gm;
    int bad = 0;
    if (i <= g.nx && j <= g.ny) {
        const bool has_u = j < g.ny, has_v = i < g.nx, cell = has_u && has_v;
        const int iw = max(i - 1, 0), ie = min(i + 1, g.nx), js = max(j - 1, 0), jn = min(j + 1, g.ny);
        const long long c = (long long)j * P + i;
        const long long cW = (long long)j * P + iw, cE = (long long)j * P + ie;
        const long long cS = (long long)js * P + i, cN = (long long)jn * P + i;
        // independent loads (clamped neighbours are used only where the face kind allows)
        const bool uk0 = g.uk[c] == FK_UNK, ukE = g.uk[cE] == FK_UNK;
        const bool vk0 = g.vk[c] == FK_UNK, vkN = g.vk[cN] == FK_UNK;
        const f2 x0v{xh[c], xl[c]}, xW{xh[cW], xl[cW]}, xE{xh[cE], xl[cE]}, xS{xh[cS], xl[cS]}, xN{xh[cN], xl[cN]};
        const f2 u0s{ush[c], usl[c]}, uEs{ush[cE], usl[cE]}, v0s{vsh[c], vsl[c]}, vNs{vsh[cN], vsl[cN]};
        const f2 gx{K.gxh, K.gxl}, gy{K.gyh, K.gyl};
        const f2 un = corrected(uk0, u0s, x0v, xW, gx);
        const f2 vn = corrected(vk0, v0s, x0v, xS, gy);
        if (has_u) {
            s.uh[off + c] = un.h;
            s.ul[off + c] = un.l;
            bad |= !isfinite(un.h) ? ENVAR_ST_NONFINITE : 0;
            bad |= (fabsf(un.h) * K.dt > K.dxf) ? ENVAR_ST_CFL : 0;
        }
        if (has_v) {
            s.vh[off + c] = vn.h;
            s.vl[off + c] = vn.l;
            bad |= !isfinite(vn.h) ? ENVAR_ST_NONFINITE : 0;
            bad |= (fabsf(vn.h) * K.dt > K.dyf) ? ENVAR_ST_CFL : 0;
        }
        if (cell && g.fluid[c]) {
            s.p[off + c] += x0v.h - xmean;
            if (want_welford && t > 0) {
                const f2 uE = corrected(ukE, uEs, xE, x0v, gx);
                const f2 vN = corrected(vkN, vNs, xN, x0v, gy);
                const f2 uc = df_scale_half(df_add(un, uE));
                const f2 vc = df_scale_half(df_add(vn, vN));
                welford2_df(uc, vc, t, s.wf + 6 * off, g.S, c);
                if (s.wd && gm != 0) {
                    // member 0's corrected cell-centred velocity from its predictor and increment,
                    // which this kernel does not modify (member 0's own block writes only u, v, p)
                    const f2 r_x0{ref.xh[c], ref.xl[c]};
                    const f2 ru = corrected(uk0, f2{ref.ush[c], ref.usl[c]}, r_x0, f2{ref.xh[cW], ref.xl[cW]}, gx);
                    const f2 ruE = corrected(ukE, f2{ref.ush[cE], ref.usl[cE]}, f2{ref.xh[cE], ref.xl[cE]}, r_x0, gx);
                    const f2 rv = corrected(vk0, f2{ref.vsh[c], ref.vsl[c]}, r_x0, f2{ref.xh[cS], ref.xl[cS]}, gy);
                    const f2 rvN = corrected(vkN, f2{ref.vsh[cN], ref.vsl[cN]}, f2{ref.xh[cN], ref.xl[cN]}, r_x0, gy);
                    const f2 du = df_sub(uc, df_scale_half(df_add(ru, ruE)));
                    const f2 dv = df_sub(vc, df_scale_half(df_add(rv, rvN)));
                    welford2_diff(du.h + du.l, dv.h + dv.l, t, s.wd + 4 * off, g.S, c);
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
            double sv[8];
            sample_sensors_mx(g, K, x0, y0, ush, usl, vsh, vsl, xh, xl, sv);
            double *dst = series + ((long long)m * g.n_window + (t - 1)) * 8;
            for (int q = 0; q < 8; ++q) dst[q] = sv[q];
        }
    }
}

void launch_correct_mx(const Grid &g, const MixConst &K, int M, const MixState &s, const MixState &ref, double x0,
                       double y0, int want_welford, double *series, const Partials &pt, MemberCtl *ctl,
                       double div_tol, long long nfluid, cudaStream_t st)
{
    dim3 blk(32, 8), grd(cdiv(g.nx + 1, 32), cdiv(g.ny + 1, 8), M);
    k_correct_mx<<<grd, blk, 0, st>>>(g, K, s, ref, x0, y0, want_welford, series, pt, ctl, div_tol, nfluid);
    count_launches(1);
}

// ---------------------------------------------------------------------------- cost
__global__ void k_plane_partial_mx(Grid g, const float *__restrict__ hi, const float *__restrict__ lo, long long mstride,
                                   double *__restrict__ part)
{
    int m = blockIdx.y;
    const float *ph = hi + (long long)m * mstride, *pl = lo + (long long)m * mstride;
    long long ncell = (long long)g.ny * g.P;
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x) {
        int i = (int)(c % g.P);
        if (i < g.nx && g.fluid[c]) acc += (double)ph[c] + (double)pl[c];
    }
    acc = block_reduce(acc, false);
    if (threadIdx.x == 0) part[(long long)m * gridDim.x + blockIdx.x] = acc;
}

void launch_plane_partial_mx(const Grid &g, int M, const float *hi, const float *lo, long long mstride, double *part,
                             int nparts, cudaStream_t st)
{
    dim3 grd(nparts, M);
    k_plane_partial_mx<<<grd, 256, 0, st>>>(g, hi, lo, mstride, part);
    count_launches(1);
}

} // namespace envar
