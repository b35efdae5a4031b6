// k_poisson.cu -- pressure-increment solve A dp = b of the projection step, batched over members.
//
// A is the masked 5-point Neumann Laplacian in finite-volume form,
//   (A x)_c = sum_{open faces f of c} c_f (x_c - x_nb),  c_f = dy/dx (x faces), dx/dy (y faces),
// a face being open iff both adjacent cells are fluid.  The solve is
//   outer (FP64):  r = b - A x  (max |r| gives the divergence dt max|r| / (dx dy) of u^{n+1});
//                  stop when max |r| <= rtol_abs, else solve A e = r approximately and x += e;
//   inner (TM):    preconditioned CG on A e = r, preconditioner = one symmetric multigrid V-cycle
//                  (red-black Gauss-Seidel pre-smoothing, black-red post-smoothing, cell-sum
//                  restriction, piecewise-constant prolongation, coarse operators with face
//                  conductance = mean of the two covered fine conductances, i.e. rediscretisation
//                  that sees partly blocked coarse faces).  Dot products accumulate in FP64.
// In MIXED mode TM = float: the multigrid and inner CG are FP32 and the outer residual keeps the
// solve exact to the FP64 tolerance (iterative refinement).  In the FP64 modes TM = double.
//
// Per-member scalars (dots, residual max) are reduced deterministically: each block writes a
// partial, and the last block to arrive (atomic ticket) sums the partials in a fixed order and
// publishes the scalar and the convergence flags in the member's control block.  Every loop is a
// fixed number of launches (graph friendly); converged members' blocks exit at once.
#include <algorithm>

#include "df64.cuh"
#include "envar_internal.cuh"
#include "res_finish.cuh"

namespace envar {

// Dot-product accumulation: FP64-accurate in both precisions -- df64 on the FP32 pipe for float
// vectors (no FP64 instruction per cell), plain FP64 for double vectors.
template <class T> struct DotAcc;
template <> struct DotAcc<float> {
    f2 v{0.f, 0.f};
    __device__ __forceinline__ void add(float a, float b) { v = df_add(v, two_prod(a, b)); }
    // a0 b0 + a1 b1 rounded once in FP32 (the pair of a lane's cells), then added exactly
    __device__ __forceinline__ void add_pair(float a0, float b0, float a1, float b1) { v = df_add_f(v, fmaf(a0, b0, a1 * b1)); }
    __device__ __forceinline__ f2 total() { return block_sum_df(v); }
};
template <> struct DotAcc<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double a, double b) { v = fma(a, b, v); }
    __device__ __forceinline__ void add_pair(double a0, double b0, double a1, double b1) { v = fma(a0, b0, fma(a1, b1, v)); }
    __device__ __forceinline__ double total() { return block_reduce(v, false); }
};

// Level-0 conductances in the vectors' precision.
template <class T> __device__ __forceinline__ T lev0_cx(const Level &L);
template <> __device__ __forceinline__ float lev0_cx<float>(const Level &L) { return L.cxf; }
template <> __device__ __forceinline__ double lev0_cx<double>(const Level &L) { return L.cx; }
template <class T> __device__ __forceinline__ T lev0_cy(const Level &L);
template <> __device__ __forceinline__ float lev0_cy<float>(const Level &L) { return L.cyf; }
template <> __device__ __forceinline__ double lev0_cy<double>(const Level &L) { return L.cy; }

// Inner CG scalars.  FP32 vectors read the FP32 copies formed once per member, alpha by the SpMV
// block that completes p^T A p (set_alpha), beta by the r^T z finisher (k_rz_finish); FP64
// vectors divide in FP64.
__device__ __forceinline__ int rz_slot(int k) { return (k & 1) ? RS_RZB : RS_RZA; }
template <class T> __device__ __forceinline__ T cg_alpha(const RedCtx &rc, int m, int k);
template <> __device__ __forceinline__ float cg_alpha<float>(const RedCtx &rc, int m, int) { return rc.red[m].fa; }
template <> __device__ __forceinline__ double cg_alpha<double>(const RedCtx &rc, int m, int k)
{
    return rc.red[m].val[rz_slot(k)] / rc.red[m].val[RS_PQ];
}
// p^T A p of iteration k complete: alpha_k = (r^T z)_k / p^T A p
__device__ __forceinline__ void set_alpha(const RedCtx &rc, int m, int k, double pq)
{
    rc.red[m].fa = (float)(rc.red[m].val[rz_slot(k)] / pq);
}
template <class T> __device__ __forceinline__ T cg_beta(const RedCtx &rc, int m, int k);
template <> __device__ __forceinline__ float cg_beta<float>(const RedCtx &rc, int m, int) { return rc.red[m].fb; }
template <> __device__ __forceinline__ double cg_beta<double>(const RedCtx &rc, int m, int k)
{
    return rc.red[m].val[rz_slot(k)] / rc.red[m].val[rz_slot(k + 1)];
}
// The dot product r^T z of the level-0 post-smoothing is left as one partial per block (no ticket:
// a block that waited for an atomic round trip at its end would hold its SM slot through it);
// k_rz_finish forms the total.  A df64 block total is stored as its float pair in the 8-byte slot,
// a double as itself (thread 0; v is the block total).
__device__ __forceinline__ void store_partial(double *p, f2 v) { *reinterpret_cast<float2 *>(p) = make_float2(v.h, v.l); }
__device__ __forceinline__ void store_partial(double *p, double v) { *p = v; }
template <class V> __device__ __forceinline__ void write_block_partial(const RedCtx &rc, int slot, int m, V v)
{
    if (threadIdx.x == 0 && threadIdx.y == 0)
        store_partial(rc.part + ((long long)slot * rc.stride + m) * rc.nblk + blockIdx.x + gridDim.x * blockIdx.y, v);
}

// ------------------------------------------------------------------------------------------------
// outer FP64 residual:  r = b - A x  (written in TM as the inner right-hand side), e = 0,
// max |r| and sum x over fluid cells.  The last block sets outer_done.
template <class TM>
__global__ void __launch_bounds__(256) k_outer_residual(Grid g, Level L0, const double *__restrict__ b,
                                                        const double *__restrict__ x, TM *__restrict__ r,
                                                        TM *__restrict__ e, RedCtx rc, MemberCtl *ctl,
                                                        double rtol_abs, int count_it)
{
    const int m = blockIdx.z;
    if (ctl[m].outer_done) return;
    const long long off = (long long)m * g.S;
    const int i0 = blockIdx.x * TILE_W, j0 = blockIdx.y * TILE_H;
    const int tid = threadIdx.x;
    double rmax = 0.0, xs = 0.0;
#pragma unroll
    for (int q = tid; q < TILE_W * TILE_H; q += TILE_THREADS) {
        int i = i0 + (q % TILE_W), j = j0 + (q / TILE_W);
        if (i >= g.nx || j >= g.ny) continue;
        long long c = (long long)j * g.P + i;
        double rv = 0.0;
        if (g.fluid[c]) {
            double xc = x[off + c];
            double cwW = L0.cwd[c], cwE = L0.cwd[c + 1], csS = L0.csd[c], csN = L0.csd[c + g.P];
            double ax = (cwW + cwE + csS + csN) * xc;
            if (cwW != 0.0) ax -= cwW * x[off + c - 1];
            if (cwE != 0.0) ax -= cwE * x[off + c + 1];
            if (csS != 0.0) ax -= csS * x[off + c - g.P];
            if (csN != 0.0) ax -= csN * x[off + c + g.P];
            rv = b[off + c] - ax;
            xs += xc;
            rmax = fmax(rmax, fabs(rv));
        }
        r[off + c] = (TM)rv;
        e[off + c] = (TM)0;
    }
    rmax = block_reduce(rmax, true);
    xs = block_reduce(xs, false);
    double tot;
    bool last1 = publish_partial(rc, RS_RMAX, m, rmax, true, &tot);
    if (last1 && threadIdx.x == 0) {
        rc.red[m].val[RS_RMAX] = tot;
        int done = (tot <= rtol_abs) ? 1 : 0;
        ctl[m].outer_done = done;
        ctl[m].inner_done = done;
        if (!done && count_it) ctl[m].outer_its += 1;
    }
    __syncthreads();
    bool last2 = publish_partial(rc, RS_XSUM, m, xs, false, &tot);
    if (last2 && threadIdx.x == 0) rc.red[m].val[RS_XSUM] = tot;
}

template <class TM>
__global__ void __launch_bounds__(256) k_outer_update(Grid g, double *__restrict__ x, const TM *__restrict__ e,
                                                      const MemberCtl *ctl)
{
    const int m = blockIdx.z;
    if (ctl[m].outer_done) return;
    const long long off = (long long)m * g.S;
    const int i0 = blockIdx.x * TILE_W, j0 = blockIdx.y * TILE_H;
#pragma unroll
    for (int q = threadIdx.x; q < TILE_W * TILE_H; q += TILE_THREADS) {
        int i = i0 + (q % TILE_W), j = j0 + (q / TILE_W);
        if (i >= g.nx || j >= g.ny) continue;
        long long c = (long long)j * g.P + i;
        if (g.fluid[c]) x[off + c] += (double)e[off + c];
    }
}

// ------------------------------------------------------------------------------------------------
// inner CG: p_new = z + beta p_old,  q = A p_new,  partial p^T q
template <class TM>
__global__ void __launch_bounds__(256) k_spmv(Grid g, Level L0, const TM *__restrict__ z, const TM *__restrict__ pold,
                                              TM *__restrict__ pnew, TM *__restrict__ q, RedCtx rc, MemberCtl *ctl,
                                              int k)
{
    const int m = blockIdx.z;
    if (ctl[m].outer_done || ctl[m].inner_done) return;
    const long long off = (long long)m * g.S;
    const TM bt = (k > 0) ? cg_beta<TM>(rc, m, k) : (TM)0;
    const int i0 = blockIdx.x * TILE_W, j0 = blockIdx.y * TILE_H;
    const TM *zm = z + off, *pm = pold + off;
    DotAcc<TM> pq;
#pragma unroll
    for (int qq = threadIdx.x; qq < TILE_W * TILE_H; qq += TILE_THREADS) {
        int i = i0 + (qq % TILE_W), j = j0 + (qq / TILE_W);
        if (i >= g.nx || j >= g.ny) continue;
        long long c = (long long)j * g.P + i;
        TM pc = (TM)0, qv = (TM)0;
        if (g.fluid[c]) {
            pc = (k > 0) ? zm[c] + bt * pm[c] : zm[c];
            const TM *cw = cw_of<TM>(L0), *cs = cs_of<TM>(L0);
            TM cwW = cw[c], cwE = cw[c + 1], csS = cs[c], csN = cs[c + g.P];
            TM acc = (cwW + cwE + csS + csN) * pc;
            if (cwW != (TM)0) acc -= cwW * ((k > 0) ? zm[c - 1] + bt * pm[c - 1] : zm[c - 1]);
            if (cwE != (TM)0) acc -= cwE * ((k > 0) ? zm[c + 1] + bt * pm[c + 1] : zm[c + 1]);
            if (csS != (TM)0) acc -= csS * ((k > 0) ? zm[c - g.P] + bt * pm[c - g.P] : zm[c - g.P]);
            if (csN != (TM)0) acc -= csN * ((k > 0) ? zm[c + g.P] + bt * pm[c + g.P] : zm[c + g.P]);
            qv = acc;
            pq.add(pc, qv);
        }
        pnew[off + c] = pc;
        q[off + c] = qv;
    }
    const auto pqt = pq.total();
    double tot;
    if (publish_partial(rc, RS_PQ, m, pqt, false, &tot) && threadIdx.x == 0) {
        rc.red[m].val[RS_PQ] = tot;
        set_alpha(rc, m, k, tot);
        if (!(tot > 0.0)) ctl[m].inner_done = 1;   // breakdown: stop this member's inner loop
    }
}

// e += alpha p,  r -= alpha q
template <class TM>
__global__ void __launch_bounds__(256) k_axpy(Grid g, TM *__restrict__ e, TM *__restrict__ r, const TM *__restrict__ p,
                                              const TM *__restrict__ q, RedCtx rc, MemberCtl *ctl, int k)
{
    const int m = blockIdx.z;
    if (ctl[m].outer_done || ctl[m].inner_done) return;
    const long long off = (long long)m * g.S;
    const TM a = cg_alpha<TM>(rc, m, k);
    const int i0 = blockIdx.x * TILE_W, j0 = blockIdx.y * TILE_H;
#pragma unroll
    for (int qq = threadIdx.x; qq < TILE_W * TILE_H; qq += TILE_THREADS) {
        int i = i0 + (qq % TILE_W), j = j0 + (qq / TILE_W);
        if (i >= g.nx || j >= g.ny) continue;
        long long c = off + (long long)j * g.P + i;
        e[c] += a * p[c];
        r[c] -= a * q[c];
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) ctl[m].inner_its += 1;
}

template <class T> struct Pair2Of;
template <> struct Pair2Of<float> { using type = float2; };
template <> struct Pair2Of<double> { using type = double2; };

// ------------------------------------------------------------------------------------------------
// Inner CG vector kernels on level 0 (used when the level has open-face bits).
//
// k_spmv0: p_new = z + beta p_old, q = A p_new and the partial p^T q.  A warp owns a 64-column
// strip of SPMV_ROWS rows, lane l the cell pair (2l, 2l+1); it walks down the strip keeping p of
// the rows below, at and above the current one in registers, takes east / west neighbours from
// the neighbouring lanes by shuffle (from memory at the strip's edges), and uses the uniform
// level-0 conductances: (A p)_c = d_c p_c - cx (p_W + p_E) - cy (p_S + p_N), closed faces having
// zero-valued neighbours (p is zero outside the fluid, as z and p_old are).
constexpr int SPMV_ROWS = 4, SPMV_WARPS = 4;

template <class T>
__global__ void __launch_bounds__(SPMV_WARPS * 32) k_spmv0(Grid g, Level L0, const T *__restrict__ z,
                                                          const T *__restrict__ pold, T *__restrict__ pnew,
                                                          T *__restrict__ q, RedCtx rc, MemberCtl *ctl, int k)
{
    using T2 = typename Pair2Of<T>::type;
    constexpr int R = SPMV_ROWS, NR = SPMV_ROWS + 2;
    const int m = blockIdx.z;
    const long long off = (long long)m * g.S;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int iL = blockIdx.x * 64 + 2 * lane;
    const bool colok = iL + 1 < g.nx;                       // nx is even
    const int j0 = (blockIdx.y * SPMV_WARPS + w) * SPMV_ROWS;
    const T *zm = z + off, *pm = pold + off;
    // every load of the warp's rows first (rows j0 - 1 .. j0 + R; z, and p for k > 0; the strip's
    // edge cells; the open-face bits): none depends on the control word or on beta
    T2 zr[NR], pr[NR];
    T zw[R], ze[R], pw[R], pe[R];
    unsigned int ob[R];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int j = j0 - 1 + r;
        zr[r] = T2{(T)0, (T)0};
        pr[r] = T2{(T)0, (T)0};
        if (colok && j >= 0 && j < g.ny) {
            const long long c = (long long)j * g.P + iL;
            zr[r] = ld_early_nc(reinterpret_cast<const T2 *>(zm + c));
            if (k > 0) pr[r] = ld_early_nc(reinterpret_cast<const T2 *>(pm + c));
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int j = j0 + r;
        zw[r] = ze[r] = pw[r] = pe[r] = (T)0;
        ob[r] = 0u;
        if (j < g.ny) {
            const long long c = (long long)j * g.P + iL;
            if (colok) ob[r] = ld_early_nc_u16(L0.open + c);
            if (lane == 0 && iL >= 1) {
                zw[r] = ld_early_nc(zm + c - 1);
                if (k > 0) pw[r] = ld_early_nc(pm + c - 1);
            }
            if (lane == 31 && iL + 2 < g.nx) {
                ze[r] = ld_early_nc(zm + c + 2);
                if (k > 0) pe[r] = ld_early_nc(pm + c + 2);
            }
        }
    }
    if (ctl[m].outer_done || ctl[m].inner_done) return;
    const T bt = (k > 0) ? cg_beta<T>(rc, m, k) : (T)0;
    const T cx = lev0_cx<T>(L0), cy = lev0_cy<T>(L0);
    auto diag = [&](unsigned int b) {
        return ((b & 1u) ? cx : (T)0) + ((b & 2u) ? cx : (T)0) + ((b & 4u) ? cy : (T)0) + ((b & 8u) ? cy : (T)0);
    };
    // p = z + beta p_old (zero outside the domain: z and p_old are zero there)
#pragma unroll
    for (int r = 0; r < NR; ++r)
        if (k > 0) zr[r] = T2{zr[r].x + bt * pr[r].x, zr[r].y + bt * pr[r].y};
    DotAcc<T> pq;
    if (j0 < g.ny) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = j0 + r;
            if (j >= g.ny) break;
            const T2 pS = zr[r], pC = zr[r + 1], pN = zr[r + 2];
            T pW = __shfl_up_sync(0xffffffffu, pC.y, 1), pE = __shfl_down_sync(0xffffffffu, pC.x, 1);
            if (lane == 0) pW = (k > 0) ? zw[r] + bt * pw[r] : zw[r];
            if (lane == 31) pE = (k > 0) ? ze[r] + bt * pe[r] : ze[r];
            if (colok) {
                const long long c = (long long)j * g.P + iL;
                const unsigned int bl = ob[r] & 15u, br = (ob[r] >> 8) & 15u;
                const T ql = bl ? diag(bl) * pC.x - cx * (pW + pC.y) - cy * (pS.x + pN.x) : (T)0;
                const T qr = br ? diag(br) * pC.y - cx * (pC.x + pE) - cy * (pS.y + pN.y) : (T)0;
                *reinterpret_cast<T2 *>(pnew + off + c) = pC;
                *reinterpret_cast<T2 *>(q + off + c) = T2{ql, qr};
                pq.add_pair(pC.x, ql, pC.y, qr);
            }
        }
    }
    const auto pqt = pq.total();
    double tot;
    if (publish_partial(rc, RS_PQ, m, pqt, false, &tot) && threadIdx.x == 0) {
        rc.red[m].val[RS_PQ] = tot;
        set_alpha(rc, m, k, tot);
        if (!(tot > 0.0)) ctl[m].inner_done = 1;   // breakdown: stop this member's inner loop
    }
}

// k_axpy4: e += alpha p, r -= alpha q over the fluid-domain rows, four values per thread (two
// aligned pairs).
template <class T>
__global__ void __launch_bounds__(128) k_axpy4(Grid g, T *__restrict__ e, T *__restrict__ r, const T *__restrict__ p,
                                              const T *__restrict__ q, RedCtx rc, MemberCtl *ctl, int k)
{
    using T2 = typename Pair2Of<T>::type;
    const int m = blockIdx.z;
    const int i = 4 * (blockIdx.x * blockDim.x + threadIdx.x), j = blockIdx.y;
    const long long c = (long long)m * g.S + (long long)j * g.P + i;
    const bool in = i < g.nx;                                // nx % 4 == 0: all four values in
    // the data first (none of it depends on the control word or on alpha)
    T2 ev[2], rv[2], pv[2], qv[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        ev[h] = rv[h] = pv[h] = qv[h] = T2{(T)0, (T)0};
        if (in) {
            ev[h] = ld_early(reinterpret_cast<const T2 *>(e + c + 2 * h));
            rv[h] = ld_early(reinterpret_cast<const T2 *>(r + c + 2 * h));
            pv[h] = ld_early_nc(reinterpret_cast<const T2 *>(p + c + 2 * h));
            qv[h] = ld_early_nc(reinterpret_cast<const T2 *>(q + c + 2 * h));
        }
    }
    if (ctl[m].outer_done || ctl[m].inner_done) return;
    const T a = cg_alpha<T>(rc, m, k);
    if (in) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            ev[h].x += a * pv[h].x; ev[h].y += a * pv[h].y;
            rv[h].x -= a * qv[h].x; rv[h].y -= a * qv[h].y;
            *reinterpret_cast<T2 *>(e + c + 2 * h) = ev[h];
            *reinterpret_cast<T2 *>(r + c + 2 * h) = rv[h];
        }
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) ctl[m].inner_its += 1;
}

// launchers: the level-0 kernels above when the level has open-face bits and nx is a multiple of 4
template <class TM>
static void launch_spmv(const Grid &g, const Level &L0, int M, const TM *z, const TM *pold, TM *pnew, TM *q,
                        const RedCtx &rc, MemberCtl *ctl, int k, cudaStream_t st)
{
    if (L0.open) {
        dim3 grd(cdiv(g.nx, 64), cdiv(g.ny, SPMV_WARPS * SPMV_ROWS), M);
        k_spmv0<TM><<<grd, SPMV_WARPS * 32, 0, st>>>(g, L0, z, pold, pnew, q, rc, ctl, k);
    } else {
        dim3 grd(cdiv(g.nx, TILE_W), cdiv(g.ny, TILE_H), M);
        k_spmv<TM><<<grd, TILE_THREADS, 0, st>>>(g, L0, z, pold, pnew, q, rc, ctl, k);
    }
}
template <class TM>
static void launch_axpy(const Grid &g, int M, TM *e, TM *r, const TM *p, const TM *q, const RedCtx &rc,
                        MemberCtl *ctl, int k, cudaStream_t st)
{
    if (g.nx % 4 == 0) {
        dim3 grd(cdiv(g.nx / 4, 128), g.ny, M);
        k_axpy4<TM><<<grd, 128, 0, st>>>(g, e, r, p, q, rc, ctl, k);
    } else {
        dim3 grd(cdiv(g.nx, TILE_W), cdiv(g.ny, TILE_H), M);
        k_axpy<TM><<<grd, TILE_THREADS, 0, st>>>(g, e, r, p, q, rc, ctl, k);
    }
}

// ------------------------------------------------------------------------------------------------
// Red-black Gauss-Seidel smoothing of one multigrid level, nsweep red-black sweep pairs per launch.
// A block owns a tile of TW x TH cells and loads it with a halo of H = 2*nsweep + 1 cells, i.e. a
// 64 x 42 region.  Each of its 384 threads owns one 7-cell column segment of the region: the cell
// values, right-hand side, inverse diagonal and face conductances (on level 0, four open-face bits)
// stay in registers; only the east / west neighbours (and the segment ends) go through shared
// memory.  Every sub-sweep updates every cell of the region except its outer ring; a cell's value
// agrees with the global sweep sequence while it lies within H - 1 - s of the tile after sub-sweep
// s, because its neighbours lie within H - s and agreed after sub-sweep s - 1.  After 2*nsweep
// sub-sweeps the tile and its first ring therefore hold exactly the values of a global red-black
// sweep sequence, which the optional restriction (residual of the tile, summed over 2x2 children)
// and the optional FP64-accurate dot product r^T z use.
enum SmoothFlags { SF_ZERO_INIT = 1, SF_PROLONG = 2, SF_RESTRICT = 4, SF_DOT = 8, SF_INIT_DOT = 16 };

struct SmoothArgs {
    Level L;              // this level
    int Pc;               // pitch of the coarse level (prolong / restrict)
    long long Sc;         // member stride of the coarse level
    int nsweep;           // red-black sweep pairs
    int order;            // 0: red then black; 1: black then red
    int flags;
    int k;                // inner iteration (for the dot slot)
};

// Thread layout: a block of 384 threads covers a 64 x 42 region (tile + halo); each thread owns a
// 7-cell column segment.  The cell values, right-hand side, inverse diagonal and face
// conductances (on level 0, four open-face bits) stay in registers; only east / west neighbours
// and the segment ends go through shared memory.
constexpr int SC_COLS = 64, SC_SEG = 6, SC_R = 7, SC_THREADS = SC_COLS * SC_SEG;
__host__ __device__ constexpr int sc_tw(int ns) { return SC_COLS - 2 * (2 * ns + 1); }
__host__ __device__ constexpr int sc_th(int ns) { return SC_SEG * SC_R - 2 * (2 * ns + 1); }

template <class T, int NS, bool BIN>
__global__ void __launch_bounds__(SC_THREADS, sizeof(T) == 4 ? 2 : 1) k_smooth(SmoothArgs sa, const T *__restrict__ f,
                                                       const T *__restrict__ ein, T *__restrict__ e,
                                                       const T *__restrict__ ec, T *__restrict__ fc, RedCtx rc,
                                                       MemberCtl *ctl, int inner_guard)
{
    constexpr int H = 2 * NS + 1, NW = SC_COLS, NH = SC_SEG * SC_R, TW = sc_tw(NS), TH = sc_th(NS);
    constexpr int SWP = NW + 1;
    __shared__ T se[NH * SWP];
    __shared__ T sr[NH * SWP];
    const int m = blockIdx.z;
    if (ctl[m].outer_done) return;
    if (inner_guard && ctl[m].inner_done) return;
    const Level &L = sa.L;
    const long long off = (long long)m * L.S;
    const int tid = threadIdx.x;
    const int a = tid % NW, b0 = (tid / NW) * SC_R;
    const int i0 = blockIdx.x * TW, j0 = blockIdx.y * TH;
    const int gi0 = i0 - H, gj0 = j0 - H;
    const int i = gi0 + a;
    // The input guess (ein) and the output (e) are different buffers: a block reads its halo from
    // cells that neighbouring blocks overwrite, so an in-place update would race.
    const T *__restrict__ fm = f + off;
    const T *__restrict__ eim = ein + off;
    T *__restrict__ em = e + off;
    const T *__restrict__ ecm = ec + (long long)m * sa.Sc;
    const T *__restrict__ cw = cw_of<T>(L);
    const T *__restrict__ cs = cs_of<T>(L);
    const uint8_t *__restrict__ opn = L.open;
    const uint8_t *__restrict__ fl = L.fluid;
    const T cx = lev0_cx<T>(L), cy = lev0_cy<T>(L);
    const bool zero = (sa.flags & SF_ZERO_INIT) != 0;
    const bool prolong = (sa.flags & SF_PROLONG) != 0;

    // face conductances: four open-face bits per cell on level 0, four values per cell elsewhere
    constexpr int NK = BIN ? 1 : SC_R;
    T ev[SC_R], fv[SC_R], iv[SC_R];
    T kw[NK], ke[NK], ks[NK], kn[NK];
    int mk[BIN ? SC_R : 1];
#define KW(r) (BIN ? ((mk[BIN ? (r) : 0] & 1) ? cx : (T)0) : kw[BIN ? 0 : (r)])
#define KE(r) (BIN ? ((mk[BIN ? (r) : 0] & 2) ? cx : (T)0) : ke[BIN ? 0 : (r)])
#define KS(r) (BIN ? ((mk[BIN ? (r) : 0] & 4) ? cy : (T)0) : ks[BIN ? 0 : (r)])
#define KN(r) (BIN ? ((mk[BIN ? (r) : 0] & 8) ? cy : (T)0) : kn[BIN ? 0 : (r)])
#pragma unroll
    for (int r = 0; r < SC_R; ++r) {
        const int j = gj0 + b0 + r;
        const bool cell = (i >= 0 && i < L.nx && j >= 0 && j < L.ny);
        const long long c = (long long)j * L.P + i;
        T w_ = 0, e_ = 0, s_ = 0, n_ = 0;
        bool act = false;
        if (BIN) {
            const int bits = cell ? (int)opn[c] : 0;
            mk[BIN ? r : 0] = bits;
            w_ = (bits & 1) ? cx : (T)0;
            e_ = (bits & 2) ? cx : (T)0;
            s_ = (bits & 4) ? cy : (T)0;
            n_ = (bits & 8) ? cy : (T)0;
            act = bits != 0;
        } else {
            if (cell) {
                w_ = cw[c]; e_ = cw[c + 1]; s_ = cs[c]; n_ = cs[c + L.P];
                act = fl[c] != 0;
            }
            kw[BIN ? 0 : r] = w_; ke[BIN ? 0 : r] = e_; ks[BIN ? 0 : r] = s_; kn[BIN ? 0 : r] = n_;
        }
        const T d = w_ + e_ + s_ + n_;
        iv[r] = (d != (T)0) ? (T)1 / d : (T)0;
        fv[r] = cell ? fm[c] : (T)0;
        T v = (cell && !zero) ? eim[c] : (T)0;
        if (cell && prolong && act) v += ecm[(long long)(j >> 1) * sa.Pc + (i >> 1)];
        ev[r] = v;
    }
#pragma unroll
    for (int r = 0; r < SC_R; ++r) se[(b0 + r) * SWP + a] = ev[r];
    __syncthreads();

#pragma unroll
    for (int s = 0; s < 2 * NS; ++s) {
        const int col = (s & 1) ^ sa.order;           // 0 = red ((i + j) even)
#pragma unroll
        for (int r = 0; r < SC_R; ++r) {
            const int b = b0 + r;
            if (b < 1 || b > NH - 2 || a < 1 || a > NW - 2) continue;
            if (((gi0 + a + gj0 + b) & 1) != col || iv[r] == (T)0) continue;
            const T eW = se[b * SWP + a - 1], eE = se[b * SWP + a + 1];
            const T eS = (r > 0) ? ev[r > 0 ? r - 1 : 0] : se[(b - 1) * SWP + a];
            const T eN = (r < SC_R - 1) ? ev[r < SC_R - 1 ? r + 1 : 0] : se[(b + 1) * SWP + a];
            const T v = iv[r] * (fv[r] + KW(r) * eW + KE(r) * eE + KS(r) * eS + KN(r) * eN);
            ev[r] = v;
            se[b * SWP + a] = v;
        }
        __syncthreads();
    }

    // write the tile interior, dot product, residual for the restriction
    const bool restrict_ = (sa.flags & SF_RESTRICT) != 0;
    DotAcc<T> dot;
#pragma unroll
    for (int r = 0; r < SC_R; ++r) {
        const int b = b0 + r;
        const int j = gj0 + b;
        const bool inner = (a >= H && a < H + TW && b >= H && b < H + TH && i < L.nx && j < L.ny);
        if (inner) {
            em[(long long)j * L.P + i] = ev[r];
            if (sa.flags & (SF_DOT | SF_INIT_DOT)) dot.add(fv[r], ev[r]);
        }
        if (restrict_) {
            T res = (T)0;
            if (inner) {
                const T eW = se[b * SWP + a - 1], eE = se[b * SWP + a + 1];
                const T eS = (r > 0) ? ev[r > 0 ? r - 1 : 0] : se[(b - 1) * SWP + a];
                const T eN = (r < SC_R - 1) ? ev[r < SC_R - 1 ? r + 1 : 0] : se[(b + 1) * SWP + a];
                const T d = KW(r) + KE(r) + KS(r) + KN(r);
                res = fv[r] - (d * ev[r] - KW(r) * eW - KE(r) * eE - KS(r) * eS - KN(r) * eN);
            }
            sr[b * SWP + a] = res;
        }
    }
    if (restrict_) {
        __syncthreads();
        for (int q = tid; q < (TW / 2) * (TH / 2); q += SC_THREADS) {
            const int qa = q % (TW / 2), qb = q / (TW / 2);
            const int I = (i0 >> 1) + qa, J = (j0 >> 1) + qb;
            if (2 * I >= L.nx || 2 * J >= L.ny) continue;
            const int bb = H + 2 * qb, aa = H + 2 * qa;
            const T sum = sr[bb * SWP + aa] + sr[bb * SWP + aa + 1] + sr[(bb + 1) * SWP + aa] + sr[(bb + 1) * SWP + aa + 1];
            fc[(long long)m * sa.Sc + (long long)J * sa.Pc + I] = sum;
        }
    }
    if (sa.flags & (SF_DOT | SF_INIT_DOT))   // (r^T z)_0 or (r^T z)_(k+1): per-block partials
        write_block_partial(rc, (sa.flags & SF_INIT_DOT) ? rz_slot(0) : rz_slot(sa.k + 1), m, dot.total());
}
#undef KW
#undef KE
#undef KS
#undef KN

// ------------------------------------------------------------------------------------------------
// Warp-row smoother (level 0, and coarser levels whose conductances fit a 16-entry table).
// On level 0 every open face has the same conductance (cx for x faces, cy for y faces) and a
// closed face always separates a fluid cell from a solid or outside cell, whose value is zero in
// every vector the solver smooths (right-hand sides and guesses are zero there and the update
// leaves a cell with no open face at zero).  The Gauss-Seidel update of a fluid cell is therefore
// e_c = (f_c + cx (e_W + e_E) + cy (e_S + e_N)) / d_c, with d_c = cx (#open x faces) +
// cy (#open y faces); a cell with no open face gets 1/d_c = 0.
//
// Layout: a block's region is 64 columns x (WARPS * R) rows; warp w owns R consecutive rows and
// lane l the cell pair (2l, 2l+1) of each: one red and one black cell per row, so a half-sweep
// updates exactly one cell per lane and row, chosen by the row's parity (the region starts on an
// even column and row).  East / west neighbours come from the neighbouring lane by shuffle,
// north / south ones from the lane's own registers, except across warps, where the boundary rows
// go through shared memory (double-buffered, one barrier per half-sweep).  The halo is
// H = 2 nsweep + 2 cells (even, for the alignment).  The region's outermost ring lacks neighbours,
// so its inverse diagonal is zeroed and it goes wrong at its first update; a wrong value moves one
// cell inward per half-sweep, so after the 2 nsweep half-sweeps the tile and its first ring still
// hold exactly the values of the global red-black sweep sequence, which the restriction and the
// dot product use.
constexpr int S0_COLS = 64;
template <class T> struct S0 {
    static constexpr int R = sizeof(T) == 4 ? 8 : 4;   // rows per warp
};
__host__ __device__ constexpr int s0_halo(int ns) { return 2 * ns + 2; }

template <class T> struct Pair2;
template <> struct Pair2<float> { using type = float2; };
template <> struct Pair2<double> { using type = double2; };

template <class T> __device__ __forceinline__ const T *ktab_of(const Level &L);
template <> __device__ __forceinline__ const float *ktab_of<float>(const Level &L) { return L.ktabf; }
template <> __device__ __forceinline__ const double *ktab_of<double>(const Level &L) { return L.ktabd; }

// CODED = false: level 0 (uniform conductances, open-face bits).  CODED = true: a coarser level
// whose face conductances are table entries: per cell a 16-bit code holds the table indices of its
// W, E, S, N faces, and the update uses them explicitly, e_c = (f_c + sum_f k_f e_f) / sum_f k_f.
template <class T, int NS, int WARPS, bool CODED, int ORDER>
__global__ void __launch_bounds__(WARPS * 32, 2) k_smoothw(SmoothArgs sa, const T *__restrict__ f,
                                                          const T *__restrict__ ein, T *__restrict__ e,
                                                          const T *__restrict__ ec, T *__restrict__ fc, RedCtx rc,
                                                          MemberCtl *ctl, int inner_guard)
{
    using T2 = typename Pair2<T>::type;
    constexpr int R = S0<T>::R, H = s0_halo(NS), NH = WARPS * R, TW = S0_COLS - 2 * H, TH = NH - 2 * H;
    static_assert(R % 2 == 0, "rows per warp come in pairs (restriction)");
    __shared__ T2 xb[2][WARPS][2][32];   // [buffer][warp][0: bottom row, 1: top row][lane]
    const int m = blockIdx.z;
    // a converged member's blocks return before any load (a group keeps iterating while its slowest
    // member does, and the loads of the others would be spent for nothing)
    if (ctl[m].outer_done) return;
    if (inner_guard && ctl[m].inner_done) return;
    const Level &L = sa.L;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i0 = blockIdx.x * TW, j0 = blockIdx.y * TH;
    const int gi0 = i0 - H, gj0 = j0 - H;
    const int iL = gi0 + 2 * lane;                              // left cell of the pair (even)
    const bool colok = (iL >= 0 && iL + 1 < L.nx);              // nx is even: a pair is all in or all out
    const long long off = (long long)m * L.S;
    const T *__restrict__ fm = f + off;
    const T *__restrict__ eim = ein + off;
    T *__restrict__ em = e + off;
    const T *__restrict__ ecm = ec + (long long)m * sa.Sc;
    const T cx = lev0_cx<T>(L), cy = lev0_cy<T>(L);
    // ORDER 0: pre-smoothing (zero guess, red first, residual restricted); ORDER 1:
    // post-smoothing (coarse correction prolonged, black first)
    constexpr bool zero = ORDER == 0, prolong = ORDER == 1;

    // CODED: conductance tables [x 0..15 | y 0..15].  Level 0: diagonal and its inverse per
    // open-face pattern (W 1, E 2, S 4, N 8).
    __shared__ T tab[32];
    if (CODED) {
        if (threadIdx.x < 32) tab[threadIdx.x] = ktab_of<T>(L)[threadIdx.x];
    } else if (threadIdx.x < 16) {
        const unsigned int q = threadIdx.x;
        const T d = ((q & 1u) ? cx : (T)0) + ((q & 2u) ? cx : (T)0) + ((q & 4u) ? cy : (T)0) + ((q & 8u) ? cy : (T)0);
        tab[q] = d;
        tab[16 + q] = (d != (T)0) ? (T)1 / d : (T)0;
    }
    __syncthreads();
    // face conductances of a cell from its code (CODED)
    auto kW = [&](unsigned int q) { return tab[q & 15u]; };
    auto kE = [&](unsigned int q) { return tab[(q >> 4) & 15u]; };
    auto kS = [&](unsigned int q) { return tab[16 + ((q >> 8) & 15u)]; };
    auto kN = [&](unsigned int q) { return tab[16 + ((q >> 12) & 15u)]; };

    T e0[R], e1[R], f0[R], f1[R], v0[R], v1[R];
    // level 0: 8 open bits (two cells) per row, 4 rows per word; CODED: both cells' codes per row
    constexpr int NB = CODED ? R : (R + 3) / 4;
    unsigned int bits[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) bits[q] = 0u;
    const long long c0 = (long long)(gj0 + w * R) * L.P + iL;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int j = gj0 + w * R + r;
        const bool ok = colok && j >= 0 && j < L.ny;
        const long long c = c0 + (long long)r * L.P;
        T2 fv = {(T)0, (T)0}, ev = {(T)0, (T)0};
        unsigned int qq = 0u, actl = 0u, actr = 0u;
        if (ok) {
            if (CODED) {
                qq = *reinterpret_cast<const unsigned int *>(L.code + c);   // left cell low half
                const unsigned int fl = *reinterpret_cast<const unsigned short *>(L.fluid + c);
                actl = fl & 0x00ffu; actr = fl & 0xff00u;
            } else {
                qq = *reinterpret_cast<const unsigned short *>(L.open + c);  // left cell low byte
                actl = qq & 0x00ffu; actr = qq & 0xff00u;
            }
            fv = *reinterpret_cast<const T2 *>(fm + c);
            if (!zero) ev = *reinterpret_cast<const T2 *>(eim + c);
            if (prolong) {
                const T cv = ecm[(long long)(j >> 1) * sa.Pc + (iL >> 1)];
                if (actl) ev.x += cv;
                if (actr) ev.y += cv;
            }
        }
        T il, ir;
        if (CODED) {
            bits[r] = qq;
            const unsigned int ql = qq & 0xffffu, qr = qq >> 16;
            const T dl = kW(ql) + kE(ql) + kS(ql) + kN(ql), dr = kW(qr) + kE(qr) + kS(qr) + kN(qr);
            il = (dl != (T)0) ? (T)1 / dl : (T)0;
            ir = (dr != (T)0) ? (T)1 / dr : (T)0;
        } else {
            const unsigned int bl = qq & 15u, br = (qq >> 8) & 15u;
            bits[r >> 2] |= (bl | (br << 4)) << ((r & 3) * 8);
            il = tab[16 + bl];
            ir = tab[16 + br];
        }
        const bool ring_row = (w == 0 && r == 0) || (w == WARPS - 1 && r == R - 1);
        v0[r] = (ring_row || lane == 0) ? (T)0 : il;
        v1[r] = (ring_row || lane == 31) ? (T)0 : ir;
        f0[r] = fv.x; f1[r] = fv.y;
        e0[r] = ev.x; e1[r] = ev.y;
    }
    xb[1][w][0][lane] = T2{e0[0], e1[0]};
    xb[1][w][1][lane] = T2{e0[R - 1], e1[R - 1]};
    __syncthreads();

    const int wb = (w > 0) ? w - 1 : 0, wa = (w < WARPS - 1) ? w + 1 : WARPS - 1;
#pragma unroll
    for (int s = 0; s < 2 * NS; ++s) {
        const int col = (s & 1) ^ ORDER;   // colour updated ((i + j) & 1 == col), known after unrolling
        const int rbuf = (s & 1) ^ 1, wbuf = s & 1;
        const T2 below = xb[rbuf][wb][1][lane];                  // top row of the warp below
        const T2 above = xb[rbuf][wa][0][lane];                  // bottom row of the warp above
#pragma unroll
        for (int r = 0; r < R; ++r) {
            // the left cell (even column) of row r has colour r & 1 (gj0 and w R are even)
            if ((r & 1) == col) {
                const T sS = (r > 0) ? e0[r > 0 ? r - 1 : 0] : below.x;
                const T sN = (r < R - 1) ? e0[r < R - 1 ? r + 1 : 0] : above.x;
                const T eW = __shfl_up_sync(0xffffffffu, e1[r], 1);
                if (CODED) {
                    const unsigned int q = bits[CODED ? r : 0] & 0xffffu;
                    e0[r] = v0[r] * (f0[r] + kW(q) * eW + kE(q) * e1[r] + kS(q) * sS + kN(q) * sN);
                } else {
                    e0[r] = v0[r] * (f0[r] + cx * (eW + e1[r]) + cy * (sS + sN));
                }
            } else {
                const T sS = (r > 0) ? e1[r > 0 ? r - 1 : 0] : below.y;
                const T sN = (r < R - 1) ? e1[r < R - 1 ? r + 1 : 0] : above.y;
                const T eE = __shfl_down_sync(0xffffffffu, e0[r], 1);
                if (CODED) {
                    const unsigned int q = bits[CODED ? r : 0] >> 16;
                    e1[r] = v1[r] * (f1[r] + kW(q) * e0[r] + kE(q) * eE + kS(q) * sS + kN(q) * sN);
                } else {
                    e1[r] = v1[r] * (f1[r] + cx * (e0[r] + eE) + cy * (sS + sN));
                }
            }
        }
        xb[wbuf][w][0][lane] = T2{e0[0], e1[0]};
        xb[wbuf][w][1][lane] = T2{e0[R - 1], e1[R - 1]};
        __syncthreads();
    }

    // tile interior: output, dot product, residual restricted to the coarse level
    constexpr int fb = (2 * NS - 1) & 1;                        // buffer of the last half-sweep
    const T2 below = xb[fb][wb][1][lane], above = xb[fb][wa][0][lane];
    const bool tile_col = colok && iL >= i0 && iL < i0 + TW;
    constexpr bool restrict_ = ORDER == 0;
    const bool want_dot = (sa.flags & (SF_DOT | SF_INIT_DOT)) != 0;
    DotAcc<T> dot;
    T racc = (T)0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int b = w * R + r, j = gj0 + b;
        const bool tile = tile_col && b >= H && b < H + TH && j < L.ny;
        const long long c = (long long)j * L.P + iL;
        if (tile) {
            *reinterpret_cast<T2 *>(em + c) = T2{e0[r], e1[r]};
            if (want_dot) dot.add_pair(f0[r], e0[r], f1[r], e1[r]);
        }
        if (restrict_) {
            const T sS0 = (r > 0) ? e0[r > 0 ? r - 1 : 0] : below.x, sN0 = (r < R - 1) ? e0[r < R - 1 ? r + 1 : 0] : above.x;
            const T sS1 = (r > 0) ? e1[r > 0 ? r - 1 : 0] : below.y, sN1 = (r < R - 1) ? e1[r < R - 1 ? r + 1 : 0] : above.y;
            const T eW = __shfl_up_sync(0xffffffffu, e1[r], 1), eE = __shfl_down_sync(0xffffffffu, e0[r], 1);
            T res0, res1;
            if (CODED) {
                // residual f - A e with the explicit conductances (zero across closed faces)
                const unsigned int ql = bits[CODED ? r : 0] & 0xffffu, qr = bits[CODED ? r : 0] >> 16;
                res0 = f0[r] - ((kW(ql) + kE(ql) + kS(ql) + kN(ql)) * e0[r] - kW(ql) * eW - kE(ql) * e1[r] -
                                kS(ql) * sS0 - kN(ql) * sN0);
                res1 = f1[r] - ((kW(qr) + kE(qr) + kS(qr) + kN(qr)) * e1[r] - kW(qr) * e0[r] - kE(qr) * eE -
                                kS(qr) * sS1 - kN(qr) * sN1);
            } else {
                // residual f - A e.  A fluid cell's closed faces have zero-valued neighbours, as in
                // the sweep; a cell with no open face has the residual f (zero in a solid cell),
                // whatever its neighbours hold.
                const unsigned int bb = bits[r >> 2] >> ((r & 3) * 8);
                const unsigned int ql = bb & 15u, qr = (bb >> 4) & 15u;
                res0 = ql ? f0[r] - (tab[ql] * e0[r] - cx * (eW + e1[r]) - cy * (sS0 + sN0)) : f0[r];
                res1 = qr ? f1[r] - (tab[qr] * e1[r] - cx * (e0[r] + eE) - cy * (sS1 + sN1)) : f1[r];
            }
            const T res = res0 + res1;
            if (r & 1) {
                if (tile) {
                    const int I = iL >> 1, J = j >> 1;
                    fc[(long long)m * sa.Sc + (long long)J * sa.Pc + I] = racc + res;
                }
            } else {
                racc = res;
            }
        }
    }
    if (want_dot)   // (r^T z)_0 or (r^T z)_(k+1): per-block partials
        write_block_partial(rc, (sa.flags & SF_INIT_DOT) ? rz_slot(0) : rz_slot(sa.k + 1), m, dot.total());
}

// ------------------------------------------------------------------------------------------------
// Coarse levels (lc .. nlev-1): one block per member runs the rest of the V-cycle in shared memory.
// Each level's face conductances and fluid flags are staged in shared memory once per launch, so
// the sweeps touch no global memory; the levels of at most COARSE_WARP_CELLS cells run in warp 0
// alone, synchronised by __syncwarp instead of block barriers.
constexpr int COARSE_WARP_CELLS = 256;

struct CoarseArgs {
    Level lev[MAX_LEVELS];
    CoarseLayout lay;
    const uint4 *img;       // the constant part of the layout, lay.image_bytes
    int lc, lw, nlev;       // first coarse level; first level run by warp 0 alone (nlev: none)
    int nu_pre, nu_post, coarse_sweeps;
    int inner_guard;
};

CoarseLayout coarse_layout(const Level *lev, int lc, int nlev, size_t tsz)
{
    CoarseLayout L{};
    auto up16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    size_t b = 0;
    for (int l = lc; l < nlev; ++l) {
        const size_t nx = lev[l].nx, ny = lev[l].ny;
        L.cw[l] = (int)b; b = up16(b + tsz * (nx + 1) * ny);
        L.cs[l] = (int)b; b = up16(b + tsz * nx * (ny + 1));
        L.fl[l] = (int)b; b = up16(b + nx * ny);
    }
    L.image_bytes = (int)b;
    for (int l = lc; l < nlev; ++l) {
        L.e[l] = (int)b;
        b = up16(b + tsz * 2 * (size_t)lev[l].nx * lev[l].ny);
    }
    L.total_bytes = (int)b;
    return L;
}

template <class T> struct CLev {
    int nx, ny;
    T *e, *f, *cw, *cs;
    uint8_t *fl;
};
template <class T> __device__ __forceinline__ CLev<T> clev(const CoarseArgs &ca, unsigned char *smem, int l)
{
    const Level &L = ca.lev[l];
    T *e = reinterpret_cast<T *>(smem + ca.lay.e[l]);
    return CLev<T>{L.nx, L.ny, e, e + L.nx * L.ny, reinterpret_cast<T *>(smem + ca.lay.cw[l]),
                   reinterpret_cast<T *>(smem + ca.lay.cs[l]), smem + ca.lay.fl[l]};
}

template <bool WARP> __device__ __forceinline__ void csync()
{
    if (WARP) __syncwarp(); else __syncthreads();
}

// Loops over a level's global rows (staging in and out): row j by warp (stride = warps in use),
// column by lane (stride 32), so no thread divides by the level's width and loads coalesce.
#define CL_ROWS(j, tid, nt, ny) for (int j = (tid) >> 5; j < (ny); j += (nt) >> 5)
#define CL_COLS(i, tid, n) for (int i = (tid) & 31; i < (n); i += 32)

// Flat loops over the cells of a level in shared memory: item t -> (row t / w, column t % w), the
// quotient by a multiply-high with m = floor((2^32 - 1) / w) + 1, exact for 2 <= w and t w < 2^32
// (coarse levels have w >= 2 cells per colour row and fewer than 2^16 cells).
__device__ __forceinline__ unsigned int div_magic(int w) { return 0xFFFFFFFFu / (unsigned int)w + 1u; }
__device__ __forceinline__ int qdiv(int t, unsigned int m) { return (int)__umulhi((unsigned int)t, m); }

// smoothing update e = acc / d: FP32 with the fast reciprocal (pre- and post-smoothing use the same
// per-cell factor, so the V-cycle stays symmetric), FP64 exact
__device__ __forceinline__ float gs_div(float a, float d) { return __fdividef(a, d); }
__device__ __forceinline__ double gs_div(double a, double d) { return a / d; }

// one Gauss-Seidel half-sweep over the cells of one colour ((i + j) & 1 == colour): every thread
// takes cells t, t + nt, ... of the colour's cells in row-major order
template <class T>
__device__ __forceinline__ void cl_sweep(const CLev<T> &L, int colour, int tid, int nt)
{
    const int hx = (L.nx + 1) >> 1;
    const unsigned int m = div_magic(hx);
    const int n = hx * L.ny;
    for (int t = tid; t < n; t += nt) {
        const int j = qdiv(t, m), i = 2 * (t - j * hx) + ((j + colour) & 1);
        if (i >= L.nx) continue;
        const int q = j * L.nx + i, w = j * (L.nx + 1) + i;
        const T cW = L.cw[w], cE = L.cw[w + 1], cS = L.cs[q], cN = L.cs[q + L.nx];
        const T d = cW + cE + cS + cN;
        if (d == (T)0) continue;
        T acc = L.f[q];
        if (i > 0) acc += cW * L.e[q - 1];
        if (i + 1 < L.nx) acc += cE * L.e[q + 1];
        if (j > 0) acc += cS * L.e[q - L.nx];
        if (j + 1 < L.ny) acc += cN * L.e[q + L.nx];
        L.e[q] = gs_div(acc, d);
    }
}

// zero guess, pre-smoothing, residual restricted (cell sums) to the next level's right-hand side
template <class T, bool WARP>
__device__ void cl_descend(const CoarseArgs &ca, unsigned char *smem, int l, int tid, int nt)
{
    const CLev<T> V = clev<T>(ca, smem, l), C = clev<T>(ca, smem, l + 1);
    for (int q = tid; q < V.nx * V.ny; q += nt) V.e[q] = (T)0;
    csync<WARP>();
    for (int s = 0; s < ca.nu_pre; ++s) {
        cl_sweep<T>(V, 0, tid, nt); csync<WARP>();
        cl_sweep<T>(V, 1, tid, nt); csync<WARP>();
    }
    const unsigned int mc = div_magic(C.nx);
    for (int t = tid; t < C.nx * C.ny; t += nt) {
        const int J = qdiv(t, mc), I = t - J * C.nx;
        T sum = (T)0;
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                const int i = 2 * I + di, j = 2 * J + dj;
                const int qq = j * V.nx + i, w = j * (V.nx + 1) + i;
                const T cW = V.cw[w], cE = V.cw[w + 1], cS = V.cs[qq], cN = V.cs[qq + V.nx];
                T ax = (cW + cE + cS + cN) * V.e[qq];
                if (i > 0) ax -= cW * V.e[qq - 1];
                if (i + 1 < V.nx) ax -= cE * V.e[qq + 1];
                if (j > 0) ax -= cS * V.e[qq - V.nx];
                if (j + 1 < V.ny) ax -= cN * V.e[qq + V.nx];
                sum += V.f[qq] - ax;
            }
        C.f[t] = sum;
    }
    csync<WARP>();
}

// coarsest level: coarse_sweeps red-black pairs, then as many black-red pairs (symmetric)
template <class T, bool WARP>
__device__ void cl_coarsest(const CoarseArgs &ca, unsigned char *smem, int l, int tid, int nt)
{
    const CLev<T> V = clev<T>(ca, smem, l);
    for (int q = tid; q < V.nx * V.ny; q += nt) V.e[q] = (T)0;
    csync<WARP>();
    for (int s = 0; s < ca.coarse_sweeps; ++s) {
        cl_sweep<T>(V, 0, tid, nt); csync<WARP>();
        cl_sweep<T>(V, 1, tid, nt); csync<WARP>();
    }
    for (int s = 0; s < ca.coarse_sweeps; ++s) {
        cl_sweep<T>(V, 1, tid, nt); csync<WARP>();
        cl_sweep<T>(V, 0, tid, nt); csync<WARP>();
    }
}

// piecewise-constant prolongation of level l+1's correction onto the fluid cells of level l,
// then post-smoothing (black-red)
template <class T, bool WARP>
__device__ void cl_ascend(const CoarseArgs &ca, unsigned char *smem, int l, int tid, int nt)
{
    const CLev<T> V = clev<T>(ca, smem, l), C = clev<T>(ca, smem, l + 1);
    const unsigned int mv = div_magic(V.nx);
    for (int q = tid; q < V.nx * V.ny; q += nt) {
        const int j = qdiv(q, mv), i = q - j * V.nx;
        if (V.fl[q]) V.e[q] += C.e[(j >> 1) * C.nx + (i >> 1)];
    }
    csync<WARP>();
    for (int s = 0; s < ca.nu_post; ++s) {
        cl_sweep<T>(V, 1, tid, nt); csync<WARP>();
        cl_sweep<T>(V, 0, tid, nt); csync<WARP>();
    }
}

template <class T>
__global__ void __launch_bounds__(1024) k_coarse(CoarseArgs ca, const T *__restrict__ fin, T *__restrict__ eout,
                                                 MemberCtl *ctl)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int m = blockIdx.x;
    if (ctl[m].outer_done) return;
    if (ca.inner_guard && ctl[m].inner_done) return;
    const int lc = ca.lc, nl = ca.nlev, tid = threadIdx.x, nt = blockDim.x;
    // constants of every coarse level: one vectorised copy of the prebuilt image; right-hand side
    // of level lc
    {
        uint4 *dst = reinterpret_cast<uint4 *>(smem);
        const int nv = ca.lay.image_bytes >> 4;
#pragma unroll 4
        for (int q = tid; q < nv; q += nt) dst[q] = ca.img[q];
        const Level &L = ca.lev[lc];
        const CLev<T> V = clev<T>(ca, smem, lc);
        CL_ROWS(j, tid, nt, L.ny) CL_COLS(i, tid, L.nx) V.f[j * L.nx + i] = fin[(long long)m * L.S + (long long)j * L.P + i];
    }
    __syncthreads();
    // block-wide levels lc .. lt-1, then the tail lt .. nl-1 (in warp 0 when its levels are small)
    const int lt = (ca.lw < nl) ? ca.lw : nl - 1;
    for (int l = lc; l < lt; ++l) cl_descend<T, false>(ca, smem, l, tid, nt);
    if (ca.lw < nl) {
        if (tid < 32) {
            for (int l = lt; l < nl - 1; ++l) cl_descend<T, true>(ca, smem, l, tid, 32);
            cl_coarsest<T, true>(ca, smem, nl - 1, tid, 32);
            for (int l = nl - 2; l >= lt; --l) cl_ascend<T, true>(ca, smem, l, tid, 32);
        }
        __syncthreads();
    } else {
        cl_coarsest<T, false>(ca, smem, nl - 1, tid, nt);
    }
    for (int l = lt - 1; l >= lc; --l) cl_ascend<T, false>(ca, smem, l, tid, nt);
    {
        const Level &L = ca.lev[lc];
        const CLev<T> V = clev<T>(ca, smem, lc);
        CL_ROWS(j, tid, nt, L.ny) CL_COLS(i, tid, L.nx) eout[(long long)m * L.S + (long long)j * L.P + i] = V.e[j * L.nx + i];
    }
}

// smoothing sweep pairs on level l: the finest level's own, or nu_c below it when set
static inline int level_sweeps(const PoissonCfg &pc, int l, int nu_finest) { return (l > 0 && pc.nu_c) ? pc.nu_c : nu_finest; }

// kernel arguments and dynamic shared memory of the coarse block
template <class T>
static size_t coarse_args(const Level *lev, const PoissonCfg &pc, int inner_guard, CoarseArgs *ca)
{
    for (int l = 0; l < pc.nlev; ++l) ca->lev[l] = lev[l];
    ca->lay = coarse_layout(lev, pc.ncoarse, pc.nlev, sizeof(T));
    ca->img = reinterpret_cast<const uint4 *>(pc.cimg);
    ca->lc = pc.ncoarse;
    ca->nlev = pc.nlev;
    ca->lw = pc.nlev;
    for (int l = pc.ncoarse; l < pc.nlev; ++l)
        if (lev[l].nx * lev[l].ny <= COARSE_WARP_CELLS) { ca->lw = l; break; }
    ca->nu_pre = level_sweeps(pc, pc.ncoarse, pc.nu_pre);
    ca->nu_post = level_sweeps(pc, pc.ncoarse, pc.nu_post);
    ca->coarse_sweeps = pc.coarse_sweeps;
    ca->inner_guard = inner_guard;
    return (size_t)ca->lay.total_bytes;
}

// ------------------------------------------------------------------------------------------------
template <class T, bool BIN>
static void launch_smooth_b(int M, int nsweep, cudaStream_t st, const SmoothArgs &sa, const T *f, const T *ein, T *e,
                            const T *ec, T *fc, const RedCtx &rc, MemberCtl *ctl, int inner_guard)
{
    const Level &L = sa.L;
    switch (nsweep) {
    case 1: {
        dim3 grd(cdiv(L.nx, sc_tw(1)), cdiv(L.ny, sc_th(1)), M);
        k_smooth<T, 1, BIN><<<grd, SC_THREADS, 0, st>>>(sa, f, ein, e, ec, fc, rc, ctl, inner_guard);
        break;
    }
    case 2: {
        dim3 grd(cdiv(L.nx, sc_tw(2)), cdiv(L.ny, sc_th(2)), M);
        k_smooth<T, 2, BIN><<<grd, SC_THREADS, 0, st>>>(sa, f, ein, e, ec, fc, rc, ctl, inner_guard);
        break;
    }
    default: {
        dim3 grd(cdiv(L.nx, sc_tw(3)), cdiv(L.ny, sc_th(3)), M);
        k_smooth<T, 3, BIN><<<grd, SC_THREADS, 0, st>>>(sa, f, ein, e, ec, fc, rc, ctl, inner_guard);
        break;
    }
    }
    count_launches(1);
}

template <class T, int NS, int WARPS, bool CODED>
static void launch_smoothw_ns(int M, cudaStream_t st, const SmoothArgs &sa, const T *f, const T *ein, T *e,
                              const T *ec, T *fc, const RedCtx &rc, MemberCtl *ctl, int inner_guard)
{
    constexpr int H = s0_halo(NS), TW = S0_COLS - 2 * H, TH = WARPS * S0<T>::R - 2 * H;
    dim3 grd(cdiv(sa.L.nx, TW), cdiv(sa.L.ny, TH), M);
    // the warp-row kernel ties the work to the order: pre-smoothing = zero guess + restriction,
    // post-smoothing = prolongation (+ optional dot), which is how the V-cycle calls it
    if (sa.order)
        k_smoothw<T, NS, WARPS, CODED, 1><<<grd, WARPS * 32, 0, st>>>(sa, f, ein, e, ec, fc, rc, ctl, inner_guard);
    else
        k_smoothw<T, NS, WARPS, CODED, 0><<<grd, WARPS * 32, 0, st>>>(sa, f, ein, e, ec, fc, rc, ctl, inner_guard);
}

// Level 0: 12 warps per block (96 x 64 regions for FP32); coded coarser levels: 8 warps.
template <class T, int WARPS, bool CODED>
static void launch_smoothw(int M, int nsweep, cudaStream_t st, const SmoothArgs &sa, const T *f, const T *ein, T *e,
                           const T *ec, T *fc, const RedCtx &rc, MemberCtl *ctl, int inner_guard)
{
    switch (nsweep) {
    case 1: launch_smoothw_ns<T, 1, WARPS, CODED>(M, st, sa, f, ein, e, ec, fc, rc, ctl, inner_guard); break;
    case 2: launch_smoothw_ns<T, 2, WARPS, CODED>(M, st, sa, f, ein, e, ec, fc, rc, ctl, inner_guard); break;
    default: launch_smoothw_ns<T, 3, WARPS, CODED>(M, st, sa, f, ein, e, ec, fc, rc, ctl, inner_guard); break;
    }
    count_launches(1);
}

template <class T>
static void launch_smooth(int M, int nsweep, cudaStream_t st, const SmoothArgs &sa, const T *f, const T *ein, T *e,
                          const T *ec, T *fc, const RedCtx &rc, MemberCtl *ctl, int inner_guard)
{
    if (sa.L.open) launch_smoothw<T, 12, false>(M, nsweep, st, sa, f, ein, e, ec, fc, rc, ctl, inner_guard);
    else if (sa.L.code) launch_smoothw<T, 8, true>(M, nsweep, st, sa, f, ein, e, ec, fc, rc, ctl, inner_guard);
    else launch_smooth_b<T, false>(M, nsweep, st, sa, f, ein, e, ec, fc, rc, ctl, inner_guard);
}

// r^T z total of each member from the level-0 post-smoothing's n block partials, one warp per
// member, in a fixed order (lane l takes partials l, l + 32, ...; lane 0's butterfly total; df64 on
// the FP32 pipe for FP32 vectors), and what hangs on it: the start value (r^T z)_0 and a breakdown
// test (init), or beta_(k+1) and the inner convergence test (r^T z)_(k+1) <= rtol2 (r^T z)_0.
// Members whose smoothing did not run (converged) are skipped.
template <class T>
__global__ void k_rz_finish(RedCtx rc, MemberCtl *ctl, int M, int n, int init, int k, double rtol2, int inner_guard)
{
    const int m = blockIdx.x, lane = threadIdx.x;
    if (m >= M) return;
    if (ctl[m].outer_done || (inner_guard && ctl[m].inner_done)) return;
    const int slot = init ? rz_slot(0) : rz_slot(k + 1);
    const double *pp = rc.part + ((long long)slot * rc.stride + m) * rc.nblk;
    double tot;
    if constexpr (sizeof(T) == 4) {
        const float2 *pf = reinterpret_cast<const float2 *>(pp);
        f2 a{0.f, 0.f};
        for (int q = lane; q < n; q += 32) {
            const float2 v = __ldcg(pf + q);
            a = df_add(a, f2{v.x, v.y});
        }
        a = warp_sum_df(a);
        tot = (lane == 0) ? df_to_d(a) : 0.0;
    } else {
        double a = 0.0;
        for (int q = lane; q < n; q += 32) a += __ldcg(pp + q);
        tot = warp_sum(a);
    }
    if (lane != 0) return;
    rc.red[m].val[slot] = tot;
    if (init) {
        rc.red[m].val[RS_RZ0] = tot;
        if (!(tot > 0.0)) ctl[m].inner_done = 1;
    } else {
        rc.red[m].fb = (float)(tot / rc.red[m].val[rz_slot(k)]);
        if (!(tot > rtol2 * rc.red[m].val[RS_RZ0])) ctl[m].inner_done = 1;   // inner convergence
    }
}

// Blocks per member of the level-0 post-smoothing launch with nu sweep pairs: the r^T z partials
// it leaves (launch_smooth: the warp-row kernel with 12 warps on a level with open-face bits, else
// the column-segment kernel).
template <class T> int rz_parts(const Level &L0, int nu)
{
    if (L0.open) {
        const int H = s0_halo(nu), TW = S0_COLS - 2 * H, TH = 12 * S0<T>::R - 2 * H;
        return cdiv(L0.nx, TW) * cdiv(L0.ny, TH);
    }
    return cdiv(L0.nx, sc_tw(nu)) * cdiv(L0.ny, sc_th(nu));
}
int rz_parts_max(const Level &L0, bool mixed)
{
    int n = 0;
    for (int nu = 1; nu <= 3; ++nu) n = std::max(n, mixed ? rz_parts<float>(L0, nu) : rz_parts<double>(L0, nu));
    return n;
}

template <class T>
static void vcycle(const Grid &g, const Level *lev, int M, const PoissonBufs &B, const PoissonCfg &pc, RedCtx rc,
                   MemberCtl *ctl, int inner_guard, int k, int init, cudaStream_t st)
{
    // level 0 input f = r (inner residual), output z
    const T *f0 = (const T *)B.r;
    T *z = (T *)B.z;
    const int lc = pc.ncoarse;
    // descend
    for (int l = 0; l < lc; ++l) {
        const Level &L = lev[l];
        const Level &Lc = lev[l + 1];
        const int nu = level_sweeps(pc, l, pc.nu_pre);
        SmoothArgs sa{L, Lc.P, Lc.S, nu, 0, SF_ZERO_INIT | SF_RESTRICT, k};
        const T *f = (l == 0) ? f0 : (const T *)B.lev_f[l];
        T *et = (T *)B.lev_t[l];     // pre-smoothed guess, read by the post-smoothing below
        launch_smooth<T>(M, nu, st, sa, f, (const T *)nullptr, et, (const T *)nullptr, (T *)B.lev_f[l + 1], rc,
                         ctl, inner_guard);
    }
    // coarse block
    {
        CoarseArgs ca;
        const size_t smem = coarse_args<T>(lev, pc, inner_guard, &ca);
        const T *fin = (lc == 0) ? f0 : (const T *)B.lev_f[lc];
        T *eout = (lc == 0) ? z : (T *)B.lev_e[lc];
        k_coarse<T><<<M, 1024, smem, st>>>(ca, fin, eout, ctl);
        count_launches(1);
    }
    // ascend
    for (int l = lc - 1; l >= 0; --l) {
        const Level &L = lev[l];
        const Level &Lc = lev[l + 1];
        int flags = SF_PROLONG;
        if (l == 0) flags |= init ? SF_INIT_DOT : SF_DOT;
        const int nu = level_sweeps(pc, l, pc.nu_post);
        SmoothArgs sa{L, Lc.P, Lc.S, nu, 1, flags, k};
        const T *f = (l == 0) ? f0 : (const T *)B.lev_f[l];
        T *e = (l == 0) ? z : (T *)B.lev_e[l];
        launch_smooth<T>(M, nu, st, sa, f, (const T *)B.lev_t[l], e, (const T *)B.lev_e[l + 1], (T *)nullptr,
                         rc, ctl, inner_guard);
    }
    // the r^T z total of the post-smoothing (one warp per member)
    k_rz_finish<T><<<M, 32, 0, st>>>(rc, ctl, M, rz_parts<T>(lev[0], pc.nu_post), init, k, pc.inner_rtol2, inner_guard);
    count_launches(1);
}

// One application of the multigrid preconditioner z = M r (level-0 arrays of every member slot).
template <class TM>
void launch_vcycle(const Grid &g, const Level *lev, int M, const PoissonBufs &B, const PoissonCfg &pc,
                   const Partials &pt, MemberCtl *ctl, cudaStream_t st)
{
    RedCtx rc = make_ctx(pt);
    vcycle<TM>(g, lev, M, B, pc, rc, ctl, 0, 0, 1, st);
}
template void launch_vcycle<float>(const Grid &, const Level *, int, const PoissonBufs &, const PoissonCfg &,
                                   const Partials &, MemberCtl *, cudaStream_t);
template void launch_vcycle<double>(const Grid &, const Level *, int, const PoissonBufs &, const PoissonCfg &,
                                    const Partials &, MemberCtl *, cudaStream_t);

template <class TM>
void prepare_poisson_kernels()
{
    cudaFuncSetAttribute(k_coarse<TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, COARSE_SMEM_MAX);
}
template void prepare_poisson_kernels<float>();
template void prepare_poisson_kernels<double>();

// Kernels run by the bodies of conditional nodes (each body's last kernel adds the body's size).
__device__ unsigned long long g_body_launches = 0;
unsigned long long conditional_body_launches()
{
    unsigned long long v = 0;
    cudaMemcpyFromSymbol(&v, g_body_launches, sizeof(v));
    return v;
}

// Loop condition of the refinement loop captured as a conditional WHILE node: run another
// refinement while some member of the group is above the tolerance and fewer than max_outer
// refinements were made in this step (reset = 1 before the loop starts the count at zero).  The
// count bounds the loop whatever the members' state.  body_kernels > 0: this launch closes a body
// of that many kernels (itself included), which is added to the device launch counter.
__global__ void k_refine_condition(MemberCtl *ctl, int M, int *count, int max_outer, int reset, int body_kernels,
                                   cudaGraphConditionalHandle handle, RedCtx rc, int finish_n, double rtol_abs)
{
    __shared__ int s_any;
    if (threadIdx.x == 0) s_any = 0;
    // the df64 residual's totals first (finish_n > 0: its block partials per member), one warp per member
    if (finish_n > 0)
        for (int m = threadIdx.x >> 5; m < M; m += blockDim.x >> 5) res_finish_member(rc, ctl, m, finish_n, rtol_abs, 1);
    __syncthreads();
    int any = 0;
    for (int m = threadIdx.x; m < M; m += blockDim.x) any |= !ctl[m].outer_done;
    if (any) atomicOr(&s_any, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        const int c = reset ? 0 : *count + 1;
        *count = c;
        cudaGraphSetConditional(handle, (s_any && c < max_outer) ? 1u : 0u);
        if (body_kernels > 0) atomicAdd(&g_body_launches, (unsigned long long)body_kernels);
    }
}

// finish: 1 forms the df64 residual's totals right after it, 0 leaves them to the condition kernel
// that follows (the FP64 residual forms its own)
template <class TM>
static void outer_residual(const Grid &g, const Level &L0, int M, const PoissonBufs &B, const PoissonCfg &pc, RedCtx rc,
                           MemberCtl *ctl, int count_it, int finish, cudaStream_t st)
{
    if (pc.df_outer) {
        launch_outer_residual_mx(g, L0, pc.mc, M, B.ms, (float *)B.r, (float *)B.e, rc, ctl, pc.rtol_abs, count_it,
                                 finish, st);
    } else {
        dim3 grd(cdiv(g.nx, TILE_W), cdiv(g.ny, TILE_H), M);
        k_outer_residual<TM><<<grd, TILE_THREADS, 0, st>>>(g, L0, B.b, B.x, (TM *)B.r, (TM *)B.e, rc, ctl, pc.rtol_abs,
                                                          count_it);
        count_launches(1);
    }
}

// One refinement: V-cycle-preconditioned inner CG on r = b - A x, then x += e.
template <class TM>
static void refinement(const Grid &g, const Level *lev, int M, const PoissonBufs &B, const PoissonCfg &pc, RedCtx rc,
                       MemberCtl *ctl, cudaStream_t st)
{
    const Level &L0 = lev[0];
    TM *r = (TM *)B.r, *e = (TM *)B.e, *z = (TM *)B.z, *q = (TM *)B.q;
    TM *pv[2] = {(TM *)B.pv, (TM *)B.pv1};
    vcycle<TM>(g, lev, M, B, pc, rc, ctl, 0, 0, 1, st);
    for (int k = 0; k < pc.max_inner; ++k) {
        launch_spmv<TM>(g, L0, M, z, pv[k & 1], pv[(k + 1) & 1], q, rc, ctl, k, st);
        count_launches(1);
        if (k + 1 == pc.max_inner && pc.df_outer) {
            // df64 x: the last update goes straight into x (x += e + alpha p), r is not needed
            launch_axpy_last_mx(g, M, B.ms, (const float *)e, (const float *)pv[(k + 1) & 1], rc, ctl, k, st);
            return;
        }
        launch_axpy<TM>(g, M, e, r, pv[(k + 1) & 1], q, rc, ctl, k, st);
        count_launches(1);
        if (k + 1 == pc.max_inner) break;   // the last update needs no new preconditioned residual
        vcycle<TM>(g, lev, M, B, pc, rc, ctl, 1, k, 0, st);   // also decides inner convergence
    }
    if (pc.df_outer) {
        return;   // max_inner == 0: nothing to add
    } else {
        dim3 grd(cdiv(g.nx, TILE_W), cdiv(g.ny, TILE_H), M);
        k_outer_update<TM><<<grd, TILE_THREADS, 0, st>>>(g, B.x, e, ctl);
        count_launches(1);
    }
}

// The pressure solve of one time step.  Inside a stream capture (the step graphs) the refinement
// loop is a conditional WHILE node whose body is one refinement and the residual after it: it
// runs as many refinements as the slowest member of the group needs (at most max_outer), with no
// launches for refinements nobody needs.  Outside a capture the loop is unrolled to max_outer
// refinements, converged members' blocks returning at once.
template <class TM>
void launch_pressure_solve(const Grid &g, const Level *lev, int M, const PoissonBufs &B, const PoissonCfg &pc,
                           const Partials &pt, MemberCtl *ctl, cudaStream_t st)
{
    RedCtx rc = make_ctx(pt);
    const Level &L0 = lev[0];
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edata = nullptr;
    size_t ndeps = 0;
    bool conditional = pc.conditional_loop && B.refine_count &&
                       cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, &edata, &ndeps) == cudaSuccess &&
                       cs == cudaStreamCaptureStatusActive;
    const int finish_n = pc.df_outer ? outer_residual_parts_mx(g) : 0;   // totals formed by the condition kernel
    if (conditional) {
        cudaGraphConditionalHandle handle;
        conditional = cudaGraphConditionalHandleCreate(&handle, graph, 0, 0) == cudaSuccess;
        if (conditional) {
            outer_residual<TM>(g, L0, M, B, pc, rc, ctl, 1, 0, st);
            k_refine_condition<<<1, 128, 0, st>>>(ctl, M, B.refine_count, pc.max_outer, 1, 0, handle, rc, finish_n,
                                                  pc.rtol_abs);
            count_launches(1);
            cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, &edata, &ndeps);
            cudaGraphNodeParams np{};
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = handle;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t node;
            cudaStream_t bs = nullptr;
            bool ok = cudaGraphAddNode(&node, graph, deps, edata, ndeps, &np) == cudaSuccess &&
                      cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies) ==
                          cudaSuccess &&
                      cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) == cudaSuccess;
            if (ok) {
                cudaGraph_t body = np.conditional.phGraph_out[0];
                ok = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                     cudaSuccess;
                if (ok) {
                    const long long c0 = captured_launches();
                    refinement<TM>(g, lev, M, B, pc, rc, ctl, bs);
                    outer_residual<TM>(g, L0, M, B, pc, rc, ctl, 1, 0, bs);
                    const int nb = (int)(captured_launches() - c0) + 1;
                    k_refine_condition<<<1, 128, 0, bs>>>(ctl, M, B.refine_count, pc.max_outer, 0, nb, handle, rc,
                                                          finish_n, pc.rtol_abs);
                    count_launches(1);
                    ok = cudaStreamEndCapture(bs, &body) == cudaSuccess;
                }
            }
            if (bs) cudaStreamDestroy(bs);
            // a conditional node without its full body could loop without end: the step graph
            // must not be instantiated then
            if (!ok) note_capture_failure();
            return;
        }
    }
    for (int o = 0; o <= pc.max_outer; ++o) {
        outer_residual<TM>(g, L0, M, B, pc, rc, ctl, o < pc.max_outer ? 1 : 0, 1, st);
        if (o == pc.max_outer) break;
        refinement<TM>(g, lev, M, B, pc, rc, ctl, st);
    }
}

template <class TM>
int launch_poisson_single(int which, const Grid &g, const Level *lev, int M, const PoissonBufs &B,
                          const PoissonCfg &pc, const Partials &pt, MemberCtl *ctl, cudaStream_t st)
{
    RedCtx rc = make_ctx(pt);
    const Level &L0 = lev[0], &L1 = lev[1];
    dim3 grd(cdiv(g.nx, TILE_W), cdiv(g.ny, TILE_H), M);
    TM *r = (TM *)B.r, *e = (TM *)B.e, *z = (TM *)B.z, *q = (TM *)B.q;
    TM *pv[2] = {(TM *)B.pv, (TM *)B.pv1};
    switch (which) {
    case 1: {
        SmoothArgs sa{L0, L1.P, L1.S, pc.nu_pre, 0, SF_ZERO_INIT | SF_RESTRICT, 0};
        launch_smooth<TM>(M, pc.nu_pre, st, sa, r, (const TM *)nullptr, (TM *)B.lev_t[0], (const TM *)nullptr,
                          (TM *)B.lev_f[1], rc, ctl, 0);
        return 0;
    }
    case 2: {
        SmoothArgs sa{L0, L1.P, L1.S, pc.nu_post, 1, SF_PROLONG | SF_DOT, 1};
        launch_smooth<TM>(M, pc.nu_post, st, sa, r, (const TM *)B.lev_t[0], z, (const TM *)B.lev_e[1], (TM *)nullptr,
                          rc, ctl, 0);
        return 0;
    }
    case 3: launch_spmv<TM>(g, L0, M, z, pv[1], pv[0], q, rc, ctl, 1, st); break;
    case 4: launch_axpy<TM>(g, M, e, r, pv[0], q, rc, ctl, 1, st); break;
    case 5:
        if (pc.df_outer) {
            launch_outer_residual_mx(g, L0, pc.mc, M, B.ms, (float *)r, (float *)e, rc, ctl, -1.0, 0, 0, st);
            return 0;
        }
        k_outer_residual<TM><<<grd, TILE_THREADS, 0, st>>>(g, L0, B.b, B.x, r, e, rc, ctl, -1.0, 0);
        break;
    case 7: {
        CoarseArgs ca;
        const size_t smem = coarse_args<TM>(lev, pc, 0, &ca);
        k_coarse<TM><<<M, 1024, smem, st>>>(ca, (const TM *)B.lev_f[pc.ncoarse], (TM *)B.lev_e[pc.ncoarse], ctl);
        break;
    }
    default: return -1;
    }
    count_launches(1);
    return 0;
}
template int launch_poisson_single<float>(int, const Grid &, const Level *, int, const PoissonBufs &,
                                          const PoissonCfg &, const Partials &, MemberCtl *, cudaStream_t);
template int launch_poisson_single<double>(int, const Grid &, const Level *, int, const PoissonBufs &,
                                           const PoissonCfg &, const Partials &, MemberCtl *, cudaStream_t);

template void launch_pressure_solve<float>(const Grid &, const Level *, int, const PoissonBufs &, const PoissonCfg &,
                                           const Partials &, MemberCtl *, cudaStream_t);
template void launch_pressure_solve<double>(const Grid &, const Level *, int, const PoissonBufs &, const PoissonCfg &,
                                            const Partials &, MemberCtl *, cudaStream_t);


} // namespace envar
