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
#include "envar_internal.cuh"

namespace envar {

struct RedCtx {
    int nblk;             // partial-producing blocks per member (level-0 tiles)
    double *part;         // [RS_COUNT][M][nblk]
    MemberRed *red;       // [M]
    int M;
};

__device__ __forceinline__ int tile_id() { return blockIdx.x + blockIdx.y * gridDim.x; }

// Publish a block partial; returns true in the (single) last block, whose thread 0 then holds
// the fixed-order total in *total (sum, or max when is_max).
__device__ bool publish_partial(const RedCtx &rc, int slot, int m, double v, bool is_max, double *total)
{
    __shared__ bool s_last;
    int tid = threadIdx.x + threadIdx.y * blockDim.x;
    double *p = rc.part + ((long long)slot * rc.M + m) * rc.nblk;
    if (tid == 0) {
        p[tile_id()] = v;
        __threadfence();
        unsigned int t = atomicAdd(&rc.red[m].cnt[slot], 1u);
        s_last = (t == (unsigned int)rc.nblk - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    if (tid < 32) {
        double acc = 0.0;
        for (int k = tid; k < rc.nblk; k += 32) {
            double w = __ldcg(p + k);
            acc = is_max ? fmax(acc, w) : acc + w;
        }
        acc = is_max ? warp_max(acc) : warp_sum(acc);
        if (tid == 0) {
            *total = acc;
            rc.red[m].cnt[slot] = 0;
        }
    }
    return true;
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
    double beta = 0.0;
    if (k > 0) {
        double rzk = rc.red[m].val[(k & 1) ? RS_RZB : RS_RZA];
        double rzp = rc.red[m].val[(k & 1) ? RS_RZA : RS_RZB];
        beta = rzk / rzp;
    }
    const TM bt = (TM)beta;
    const int i0 = blockIdx.x * TILE_W, j0 = blockIdx.y * TILE_H;
    const TM *zm = z + off, *pm = pold + off;
    double pq = 0.0;
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
            pq += (double)pc * (double)qv;
        }
        pnew[off + c] = pc;
        q[off + c] = qv;
    }
    pq = block_reduce(pq, false);
    double tot;
    if (publish_partial(rc, RS_PQ, m, pq, false, &tot) && threadIdx.x == 0) {
        rc.red[m].val[RS_PQ] = tot;
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
    const double alpha = rc.red[m].val[(k & 1) ? RS_RZB : RS_RZA] / rc.red[m].val[RS_PQ];
    const TM a = (TM)alpha;
    const int i0 = blockIdx.x * TILE_W, j0 = blockIdx.y * TILE_H;
    for (int qq = threadIdx.x; qq < TILE_W * TILE_H; qq += TILE_THREADS) {
        int i = i0 + (qq % TILE_W), j = j0 + (qq / TILE_W);
        if (i >= g.nx || j >= g.ny) continue;
        long long c = off + (long long)j * g.P + i;
        e[c] += a * p[c];
        r[c] -= a * q[c];
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) ctl[m].inner_its += 1;
}

// ------------------------------------------------------------------------------------------------
// Tiled red-black Gauss-Seidel on one level.  The tile (TW x TH cells) is loaded with a halo of
// H = 2*nsweep + 1 cells; sub-sweep s (0 .. 2 nsweep - 1) updates its colour on cells within
// distance H - 1 - s of the tile interior, so after all sub-sweeps the interior and its first
// ring hold exactly the values of a global red-black sweep sequence.
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

template <class T>
__device__ __forceinline__ int cell_dist(int a, int b, int H, int TW, int TH)
{
    int d = 0;
    d = max(d, H - a);
    d = max(d, a - (H + TW - 1));
    d = max(d, H - b);
    d = max(d, b - (H + TH - 1));
    return d;
}

template <class T, int TW, int TH>
__global__ void __launch_bounds__(256) k_smooth(SmoothArgs sa, const T *__restrict__ f, T *__restrict__ e,
                                                const T *__restrict__ ec, T *__restrict__ fc, RedCtx rc,
                                                MemberCtl *ctl, int inner_guard)
{
    extern __shared__ unsigned char smem_raw[];
    const int m = blockIdx.z;
    if (ctl[m].outer_done) return;
    if (inner_guard && ctl[m].inner_done) return;
    const Level &L = sa.L;
    const int H = 2 * sa.nsweep + 1;
    const int SW = TW + 2 * H + 1, SH = TH + 2 * H + 1;
    T *se = reinterpret_cast<T *>(smem_raw);
    T *sf = se + SW * SH;
    T *scw = sf + SW * SH;
    T *scs = scw + SW * SH;
    const long long off = (long long)m * L.S;
    const int i0 = blockIdx.x * TW, j0 = blockIdx.y * TH;
    const int gi0 = i0 - H, gj0 = j0 - H;
    const T *cw = cw_of<T>(L), *cs = cs_of<T>(L);
    const int tid = threadIdx.x;
    const bool zero = (sa.flags & SF_ZERO_INIT) != 0;
    const bool prolong = (sa.flags & SF_PROLONG) != 0;

    for (int q = tid; q < SW * SH; q += blockDim.x) {
        int a = q % SW, b = q / SW;
        int i = gi0 + a, j = gj0 + b;
        T vw = (T)0, vs = (T)0, ve = (T)0, vf = (T)0;
        if (i >= 0 && j >= 0) {
            long long c = (long long)j * L.P + i;
            if (j < L.ny && i <= L.nx) vw = cw[c];
            if (i < L.nx && j <= L.ny) vs = cs[c];
            if (i < L.nx && j < L.ny) {
                vf = f[off + c];
                if (!zero) ve = e[off + c];
                if (prolong && L.fluid[c]) ve += ec[(long long)m * sa.Sc + (long long)(j >> 1) * sa.Pc + (i >> 1)];
            }
        }
        scw[q] = vw;
        scs[q] = vs;
        sf[q] = vf;
        se[q] = ve;
    }
    __syncthreads();

    const int NW = TW + 2 * H, NH = TH + 2 * H;
    for (int s = 0; s < 2 * sa.nsweep; ++s) {
        const int colour = ((s & 1) ^ sa.order);          // 0 = red ((i+j) even)
        const int lim = H - 1 - s;
        for (int q = tid; q < NW * NH; q += blockDim.x) {
            int a = q % NW, b = q / NW;
            int i = gi0 + a, j = gj0 + b;
            if (((i + j) & 1) != colour) continue;
            if (cell_dist<T>(a, b, H, TW, TH) > lim) continue;
            int sq = b * SW + a;
            T cW = scw[sq], cE = scw[sq + 1], cS = scs[sq], cN = scs[sq + SW];
            T d = cW + cE + cS + cN;
            if (d == (T)0) continue;
            T acc = sf[sq] + cW * se[sq - 1] + cE * se[sq + 1] + cS * se[sq - SW] + cN * se[sq + SW];
            se[sq] = acc / d;
        }
        __syncthreads();
    }

    // write the interior
    double dot = 0.0;
    for (int q = tid; q < TW * TH; q += blockDim.x) {
        int a = H + q % TW, b = H + q / TW;
        int i = i0 + q % TW, j = j0 + q / TW;
        if (i >= L.nx || j >= L.ny) continue;
        int sq = b * SW + a;
        e[off + (long long)j * L.P + i] = se[sq];
        if (sa.flags & (SF_DOT | SF_INIT_DOT)) dot += (double)sf[sq] * (double)se[sq];
    }
    if (sa.flags & SF_RESTRICT) {
        // residual of the interior cells, summed over 2x2 children into the coarse right-hand side
        for (int q = tid; q < (TW / 2) * (TH / 2); q += blockDim.x) {
            int qa = q % (TW / 2), qb = q / (TW / 2);
            int I = (i0 >> 1) + qa, J = (j0 >> 1) + qb;
            if (2 * I >= L.nx || 2 * J >= L.ny) continue;
            T sum = (T)0;
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    int a = H + 2 * qa + di, b = H + 2 * qb + dj;
                    int sq = b * SW + a;
                    T cW = scw[sq], cE = scw[sq + 1], cS = scs[sq], cN = scs[sq + SW];
                    T ax = (cW + cE + cS + cN) * se[sq] - cW * se[sq - 1] - cE * se[sq + 1] - cS * se[sq - SW] -
                           cN * se[sq + SW];
                    sum += sf[sq] - ax;
                }
            fc[(long long)m * sa.Sc + (long long)J * sa.Pc + I] = sum;
        }
    }
    if (sa.flags & (SF_DOT | SF_INIT_DOT)) {
        dot = block_reduce(dot, false);
        double tot;
        int slot = (sa.flags & SF_INIT_DOT) ? RS_RZA : (((sa.k + 1) & 1) ? RS_RZB : RS_RZA);
        if (publish_partial(rc, slot, m, dot, false, &tot) && threadIdx.x == 0) {
            rc.red[m].val[slot] = tot;
            if (sa.flags & SF_INIT_DOT) {
                rc.red[m].val[RS_RZ0] = tot;
                if (!(tot > 0.0)) ctl[m].inner_done = 1;
            }
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Coarse levels (lc .. nlev-1): one block per member runs the rest of the V-cycle in shared memory.
struct CoarseArgs {
    Level lev[MAX_LEVELS];
    int off[MAX_LEVELS];   // smem offsets (elements) of level l's e; f follows at + nx*ny
    int lc, nlev;
    int nu_pre, nu_post, coarse_sweeps;
    int inner_guard;
};

template <class T>
__device__ void coarse_sweep(const Level &L, T *se, const T *sf, int colour)
{
    const T *cw = cw_of<T>(L), *cs = cs_of<T>(L);
    const int n = L.nx * L.ny;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        int i = q % L.nx, j = q / L.nx;
        if (((i + j) & 1) != colour) continue;
        long long c = (long long)j * L.P + i;
        T cW = cw[c], cE = cw[c + 1], cS = cs[c], cN = cs[c + L.P];
        T d = cW + cE + cS + cN;
        if (d == (T)0) continue;
        T acc = sf[q];
        if (i > 0) acc += cW * se[q - 1];
        if (i + 1 < L.nx) acc += cE * se[q + 1];
        if (j > 0) acc += cS * se[q - L.nx];
        if (j + 1 < L.ny) acc += cN * se[q + L.nx];
        se[q] = acc / d;
    }
    __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(1024) k_coarse(CoarseArgs ca, const T *__restrict__ fin, T *__restrict__ eout,
                                                 MemberCtl *ctl)
{
    extern __shared__ unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int m = blockIdx.x;
    if (ctl[m].outer_done) return;
    if (ca.inner_guard && ctl[m].inner_done) return;
    const int lc = ca.lc, nl = ca.nlev;
    {   // load f of level lc
        const Level &L = ca.lev[lc];
        T *sf = sm + ca.off[lc] + L.nx * L.ny;
        for (int q = threadIdx.x; q < L.nx * L.ny; q += blockDim.x) {
            int i = q % L.nx, j = q / L.nx;
            sf[q] = fin[(long long)m * L.S + (long long)j * L.P + i];
        }
        __syncthreads();
    }
    for (int l = lc; l < nl; ++l) {
        const Level &L = ca.lev[l];
        T *se = sm + ca.off[l];
        T *sf = se + L.nx * L.ny;
        for (int q = threadIdx.x; q < L.nx * L.ny; q += blockDim.x) se[q] = (T)0;
        __syncthreads();
        if (l == nl - 1) {
            for (int s = 0; s < ca.coarse_sweeps; ++s) { coarse_sweep<T>(L, se, sf, 0); coarse_sweep<T>(L, se, sf, 1); }
            for (int s = 0; s < ca.coarse_sweeps; ++s) { coarse_sweep<T>(L, se, sf, 1); coarse_sweep<T>(L, se, sf, 0); }
            break;
        }
        for (int s = 0; s < ca.nu_pre; ++s) { coarse_sweep<T>(L, se, sf, 0); coarse_sweep<T>(L, se, sf, 1); }
        // residual -> restriction
        const Level &Lc = ca.lev[l + 1];
        T *sfc = sm + ca.off[l + 1] + Lc.nx * Lc.ny;
        const T *cw = cw_of<T>(L), *cs = cs_of<T>(L);
        for (int q = threadIdx.x; q < Lc.nx * Lc.ny; q += blockDim.x) {
            int I = q % Lc.nx, J = q / Lc.nx;
            T sum = (T)0;
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    int i = 2 * I + di, j = 2 * J + dj;
                    int qq = j * L.nx + i;
                    long long c = (long long)j * L.P + i;
                    T cW = cw[c], cE = cw[c + 1], cS = cs[c], cN = cs[c + L.P];
                    T ax = (cW + cE + cS + cN) * se[qq];
                    if (i > 0) ax -= cW * se[qq - 1];
                    if (i + 1 < L.nx) ax -= cE * se[qq + 1];
                    if (j > 0) ax -= cS * se[qq - L.nx];
                    if (j + 1 < L.ny) ax -= cN * se[qq + L.nx];
                    sum += sf[qq] - ax;
                }
            sfc[q] = sum;
        }
        __syncthreads();
    }
    for (int l = nl - 2; l >= lc; --l) {
        const Level &L = ca.lev[l], &Lc = ca.lev[l + 1];
        T *se = sm + ca.off[l];
        T *sf = se + L.nx * L.ny;
        const T *sec = sm + ca.off[l + 1];
        for (int q = threadIdx.x; q < L.nx * L.ny; q += blockDim.x) {
            int i = q % L.nx, j = q / L.nx;
            if (L.fluid[(long long)j * L.P + i]) se[q] += sec[(j >> 1) * Lc.nx + (i >> 1)];
        }
        __syncthreads();
        for (int s = 0; s < ca.nu_post; ++s) { coarse_sweep<T>(L, se, sf, 1); coarse_sweep<T>(L, se, sf, 0); }
    }
    {
        const Level &L = ca.lev[lc];
        const T *se = sm + ca.off[lc];
        for (int q = threadIdx.x; q < L.nx * L.ny; q += blockDim.x) {
            int i = q % L.nx, j = q / L.nx;
            eout[(long long)m * L.S + (long long)j * L.P + i] = se[q];
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Inner convergence flag after the V-cycle's dot: set by a one-warp kernel per member.
__global__ void k_inner_check(RedCtx rc, MemberCtl *ctl, int k, double rtol2)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= rc.M) return;
    if (ctl[m].outer_done || ctl[m].inner_done) return;
    double rz = rc.red[m].val[((k + 1) & 1) ? RS_RZB : RS_RZA];
    if (!(rz > rtol2 * rc.red[m].val[RS_RZ0])) ctl[m].inner_done = 1;
}

// ------------------------------------------------------------------------------------------------
template <class T>
static size_t smooth_smem(int nsweep)
{
    int H = 2 * nsweep + 1;
    return sizeof(T) * 4 * (size_t)(TILE_W + 2 * H + 1) * (TILE_H + 2 * H + 1);
}

template <class T>
static void vcycle(const Grid &g, const Level *lev, int M, const PoissonBufs &B, const PoissonCfg &pc, RedCtx rc,
                   MemberCtl *ctl, int inner_guard, int k, int init, cudaStream_t st)
{
    // level 0 input f = r (inner residual), output z
    const T *f0 = (const T *)B.r;
    T *z = (T *)B.z;
    const int lc = pc.ncoarse;
    auto grid_of = [&](const Level &L) { return dim3(cdiv(L.nx, TILE_W), cdiv(L.ny, TILE_H), M); };
    // descend
    for (int l = 0; l < lc; ++l) {
        const Level &L = lev[l];
        const Level &Lc = lev[l + 1];
        SmoothArgs sa{L, Lc.P, Lc.S, pc.nu_pre, 0, SF_ZERO_INIT | SF_RESTRICT, k};
        const T *f = (l == 0) ? f0 : (const T *)B.lev_f[l];
        T *e = (l == 0) ? z : (T *)B.lev_e[l];
        k_smooth<T, TILE_W, TILE_H><<<grid_of(L), TILE_THREADS, smooth_smem<T>(pc.nu_pre), st>>>(
            sa, f, e, nullptr, (T *)B.lev_f[l + 1], rc, ctl, inner_guard);
        count_launches(1);
    }
    // coarse block
    {
        CoarseArgs ca;
        int off = 0;
        for (int l = 0; l < pc.nlev; ++l) {
            ca.lev[l] = lev[l];
            if (l >= lc) {
                ca.off[l] = off;
                off += 2 * lev[l].nx * lev[l].ny;
            } else {
                ca.off[l] = 0;
            }
        }
        ca.lc = lc;
        ca.nlev = pc.nlev;
        ca.nu_pre = pc.nu_pre;
        ca.nu_post = pc.nu_post;
        ca.coarse_sweeps = pc.coarse_sweeps;
        ca.inner_guard = inner_guard;
        const T *fin = (lc == 0) ? f0 : (const T *)B.lev_f[lc];
        T *eout = (lc == 0) ? z : (T *)B.lev_e[lc];
        k_coarse<T><<<M, 1024, sizeof(T) * off, st>>>(ca, fin, eout, ctl);
        count_launches(1);
    }
    // ascend
    for (int l = lc - 1; l >= 0; --l) {
        const Level &L = lev[l];
        const Level &Lc = lev[l + 1];
        int flags = SF_PROLONG;
        if (l == 0) flags |= init ? SF_INIT_DOT : SF_DOT;
        SmoothArgs sa{L, Lc.P, Lc.S, pc.nu_post, 1, flags, k};
        const T *f = (l == 0) ? f0 : (const T *)B.lev_f[l];
        T *e = (l == 0) ? z : (T *)B.lev_e[l];
        k_smooth<T, TILE_W, TILE_H><<<grid_of(L), TILE_THREADS, smooth_smem<T>(pc.nu_post), st>>>(
            sa, f, e, (const T *)B.lev_e[l + 1], nullptr, rc, ctl, inner_guard);
        count_launches(1);
    }
}

static RedCtx make_ctx(const Partials &pt, int M)
{
    RedCtx rc;
    rc.nblk = pt.nblk;
    rc.part = pt.part;
    rc.red = pt.red;
    rc.M = M;
    return rc;
}

template <class TM>
void prepare_poisson_kernels()
{
    cudaFuncSetAttribute(k_smooth<TM, TILE_W, TILE_H>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    cudaFuncSetAttribute(k_coarse<TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
}
template void prepare_poisson_kernels<float>();
template void prepare_poisson_kernels<double>();

template <class TM>
void launch_pressure_solve(const Grid &g, const Level *lev, int M, const PoissonBufs &B, const PoissonCfg &pc,
                           const Partials &pt, MemberCtl *ctl, cudaStream_t st)
{
    RedCtx rc = make_ctx(pt, M);
    const Level &L0 = lev[0];
    dim3 grd(cdiv(g.nx, TILE_W), cdiv(g.ny, TILE_H), M);
    TM *r = (TM *)B.r, *e = (TM *)B.e, *z = (TM *)B.z, *q = (TM *)B.q;
    TM *pv[2] = {(TM *)B.pv, (TM *)B.pv + (size_t)g.S * M};
    for (int o = 0; o <= pc.max_outer; ++o) {
        k_outer_residual<TM><<<grd, TILE_THREADS, 0, st>>>(g, L0, B.b, B.x, r, e, rc, ctl, pc.rtol_abs,
                                                          o < pc.max_outer ? 1 : 0);
        count_launches(1);
        if (o == pc.max_outer) break;
        vcycle<TM>(g, lev, M, B, pc, rc, ctl, 0, 0, 1, st);
        for (int k = 0; k < pc.max_inner; ++k) {
            k_spmv<TM><<<grd, TILE_THREADS, 0, st>>>(g, L0, z, pv[k & 1], pv[(k + 1) & 1], q, rc, ctl, k);
            k_axpy<TM><<<grd, TILE_THREADS, 0, st>>>(g, e, r, pv[(k + 1) & 1], q, rc, ctl, k);
            count_launches(2);
            if (k + 1 == pc.max_inner) break;   // the last update needs no new preconditioned residual
            vcycle<TM>(g, lev, M, B, pc, rc, ctl, 1, k, 0, st);
            k_inner_check<<<cdiv(M, 32), 32, 0, st>>>(rc, ctl, k, pc.inner_rtol2);
            count_launches(1);
        }
        k_outer_update<TM><<<grd, TILE_THREADS, 0, st>>>(g, B.x, e, ctl);
        count_launches(1);
    }
}

template <class TM>
int launch_poisson_single(int which, const Grid &g, const Level *lev, int M, const PoissonBufs &B,
                          const PoissonCfg &pc, const Partials &pt, MemberCtl *ctl, cudaStream_t st)
{
    RedCtx rc = make_ctx(pt, M);
    const Level &L0 = lev[0], &L1 = lev[1];
    dim3 grd(cdiv(g.nx, TILE_W), cdiv(g.ny, TILE_H), M);
    TM *r = (TM *)B.r, *e = (TM *)B.e, *z = (TM *)B.z, *q = (TM *)B.q;
    TM *pv[2] = {(TM *)B.pv, (TM *)B.pv + (size_t)g.S * M};
    switch (which) {
    case 1: {
        SmoothArgs sa{L0, L1.P, L1.S, pc.nu_pre, 0, SF_ZERO_INIT | SF_RESTRICT, 0};
        k_smooth<TM, TILE_W, TILE_H><<<grd, TILE_THREADS, smooth_smem<TM>(pc.nu_pre), st>>>(
            sa, r, z, nullptr, (TM *)B.lev_f[1], rc, ctl, 0);
        break;
    }
    case 2: {
        SmoothArgs sa{L0, L1.P, L1.S, pc.nu_post, 1, SF_PROLONG | SF_DOT, 1};
        k_smooth<TM, TILE_W, TILE_H><<<grd, TILE_THREADS, smooth_smem<TM>(pc.nu_post), st>>>(
            sa, r, z, (const TM *)B.lev_e[1], nullptr, rc, ctl, 0);
        break;
    }
    case 3: k_spmv<TM><<<grd, TILE_THREADS, 0, st>>>(g, L0, z, pv[1], pv[0], q, rc, ctl, 1); break;
    case 4: k_axpy<TM><<<grd, TILE_THREADS, 0, st>>>(g, e, r, pv[0], q, rc, ctl, 1); break;
    case 5: k_outer_residual<TM><<<grd, TILE_THREADS, 0, st>>>(g, L0, B.b, B.x, r, e, rc, ctl, -1.0, 0); break;
    case 7: {
        PoissonCfg p2 = pc;
        CoarseArgs ca;
        int off = 0;
        for (int l = 0; l < pc.nlev; ++l) {
            ca.lev[l] = lev[l];
            ca.off[l] = (l >= pc.ncoarse) ? off : 0;
            if (l >= pc.ncoarse) off += 2 * lev[l].nx * lev[l].ny;
        }
        ca.lc = p2.ncoarse; ca.nlev = p2.nlev; ca.nu_pre = p2.nu_pre; ca.nu_post = p2.nu_post;
        ca.coarse_sweeps = p2.coarse_sweeps; ca.inner_guard = 0;
        k_coarse<TM><<<M, 1024, sizeof(TM) * off, st>>>(ca, (const TM *)B.lev_f[p2.ncoarse], (TM *)B.lev_e[p2.ncoarse],
                                                        ctl);
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
