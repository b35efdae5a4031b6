// envar_internal.cuh -- device-side data structures and helpers of the GB300 EnVar library.
//
// Memory layout (all per-member arrays, all levels):
//   a field of a level with nx x ny cells is stored row-major with a pitch P
//   (P = nx + 1 rounded up to 32 elements) and (ny + 1) rows, so that cell
//   arrays, u-face arrays ((nx+1) x ny) and v-face arrays (nx x (ny+1)) share
//   one index  idx = j * P + i  and one member stride S = (ny + 1) * P.
//   Member m of an array starts at base + m * S.  Members are contiguous, so a
//   launch over all members is one contiguous sweep of HBM.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace envar {

// FK_SOLID faces take the odd mirror of their fluid-side neighbour inside stencils (no slip),
// FK_SLIP faces the even one (free slip: the slip segments of the lower wall).
enum FaceKind : uint8_t { FK_ZERO = 0, FK_UNK = 1, FK_INLET = 2, FK_OUTLET = 3, FK_SOLID = 4, FK_SLIP = 5 };

constexpr int MAX_LEVELS = 12;
// Level-0 tile of the Poisson / stencil kernels: 64 x 16 cells per 256-thread block.
constexpr int TILE_W = 64;
constexpr int TILE_H = 16;
constexpr int TILE_THREADS = 256;
// The coarsest levels are solved by one block per member in shared memory: from the first level
// whose levels fit COARSE_SMEM_MAX bytes (values, guesses, conductances and fluid flags).
constexpr int COARSE_SMEM_MAX = 200 * 1024;

struct Level {
    int nx, ny, P;          // cells, pitch
    long long S;            // member stride (elements)
    const uint8_t *fluid;   // [ny][P]
    const float *cwf;       // west-face conductance (i in 0..nx), [ny][P]
    const float *csf;       // south-face conductance (j in 0..ny), [ny+1][P]
    const double *cwd;
    const double *csd;
    const uint8_t *open;    // level 0 only: open-face bits (1 W, 2 E, 4 S, 8 N) of fluid cells
    double cx, cy;          // level 0 only: conductance of an open x / y face
    float cxf, cyf;         // level 0 only: the same in FP32
    // levels >= 1 with at most 16 distinct conductances per direction: per cell the table indices
    // of its W, E, S, N faces (4 bits each, W lowest) and the tables [x faces 0..15 | y faces 0..15]
    const uint16_t *code;
    const float *ktabf;
    const double *ktabd;
};

struct Grid {
    int nx, ny, P;
    long long S;
    double dx, dy, dt, nu;
    double cx, cy;          // finite-volume conductances dy/dx and dx/dy
    double hxy;             // dx * dy
    const uint8_t *fluid;   // [ny][P]
    const uint8_t *uk;      // u-face kinds [ny][P]
    const uint8_t *vk;      // v-face kinds [ny+1][P]
    const double *u_in;     // inlet profile per row
    int ia, ja, nrx, nry;   // control rectangle (cells)
    int n_steps, n_window;
    double conv_speed;
};

// Per-member control block in device memory.
struct MemberCtl {
    int step;               // completed time steps of the current forward run
    int status;             // ENVAR_ST_* bits
    int gidx;               // ensemble member held by this slot (0 = the unperturbed run)
    int pad_;
    int outer_done;         // pressure solve converged for the current step
    int inner_done;         // inner CG converged for the current refinement
    double max_div;         // max |D u| seen over the run
    long long outer_its;    // refinements performed (summed over steps)
    long long inner_its;    // inner CG iterations performed
};

// Per-member scalars of the pressure solve, reduced deterministically: every level-0 tile writes
// a partial and the last tile to arrive sums them in a fixed order into val[slot].
enum RedSlot { RS_RMAX = 0, RS_XSUM = 1, RS_RZ0 = 2, RS_RZA = 3, RS_RZB = 4, RS_PQ = 5, RS_COUNT = 6 };
struct MemberRed {
    unsigned int cnt[RS_COUNT];   // arrival tickets
    double val[RS_COUNT];         // max |r| (outer residual), sum x, r^T z (start, ping, pong), p^T A p
    // FP32 inner CG: alpha = (r^T z)_k / p^T A p and beta = (r^T z)_k / (r^T z)_(k-1), each formed
    // once per member (a double division in every thread would occupy the FP64 pipe, about 1/64 of
    // the FP32 rate, for longer than the kernel's memory traffic)
    float fa, fb;
};
struct Partials {
    int nblk;               // partial slots per member (>= blocks per member of any producing kernel)
    double *part;           // [RS_COUNT][stride][nblk]
    MemberRed *red;         // [stride]
    int stride;             // member slots of the handle (a member group's view keeps it)
};

// Mixed-precision (ENVAR_MIXED) member state: df64 quantities are hi/lo float planes.
struct MixState {
    float *uh, *ul, *vh, *vl;       // velocity u^n, v^n (df64)
    float *ush, *usl, *vsh, *vsl;   // predictor u*, v* (df64)
    float *p;                       // pressure (FP32)
    float *Ru, *Rv;                 // tendencies (FP32, AB2), two buffers each: +0 and +rstride
    long long rstride;              // offset of the second tendency buffer (elements)
    float *bh, *bl, *xh, *xl;       // Poisson right-hand side and solution (df64)
    float *xp;                      // previous pressure increment, re-centred (FP32; guess extrapolation)
    float *wf;                      // Welford per member: 6 planes (mean_u, mean_v, M2; hi/lo)
    float *wd;                      // Welford of d = u - u_0 per member: 4 planes (mean_du, mean_dv, M2 hi/lo)
    float *frect;                   // member forcing on the control rectangle (FP32)
};
// Constants of the mixed step; df64 pairs (h, l) where FP64-level accuracy is needed.
struct MixConst {
    float gxh, gxl, gyh, gyl;       // gamma = dt/dx, dt/dy       (velocity correction)
    float kxh, kxl, kyh, kyl;       // kappa = dy/dt, dx/dt       (right-hand side)
    float cxh, cxl, cyh, cyl;       // c = kappa * gamma         (Poisson operator)
    float dt, gxf, gyf, i4dx, i4dy, nudx2, nudy2, dxf, dyf;
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum / max (blockDim.x * blockDim.y threads, multiple of 32, <= 1024).
// Result valid in every thread.  Uses 33 doubles of shared memory.
__device__ __forceinline__ double block_reduce(double v, bool is_max)
{
    __shared__ double red[33];
    int t = threadIdx.x + threadIdx.y * blockDim.x;
    int nt = blockDim.x * blockDim.y;
    v = is_max ? warp_max(v) : warp_sum(v);
    __syncthreads();
    if ((t & 31) == 0) red[t >> 5] = v;
    __syncthreads();
    if (t < 32) {
        double w = (t < (nt >> 5)) ? red[t] : (is_max ? -1.0 : 0.0);
        w = is_max ? warp_max(w) : warp_sum(w);
        if (t == 0) red[32] = w;
    }
    __syncthreads();
    double r = red[32];
    __syncthreads();
    return r;
}

// Sum (or max) of a member's partials in a fixed order -- every block that calls
// this gets the bit-identical result.  Called by whole warps; result in all lanes.
__device__ __forceinline__ double warp_partials(const double *p, int n, bool is_max)
{
    int lane = threadIdx.x & 31;
    double v = is_max ? 0.0 : 0.0;
    for (int k = lane; k < n; k += 32) v = is_max ? fmax(v, p[k]) : v + p[k];
    return is_max ? warp_max(v) : warp_sum(v);
}

struct RedCtx {
    int nblk;             // partial slots per member (capacity)
    double *part;         // [RS_COUNT][stride][nblk]
    MemberRed *red;       // [stride]
    int stride;
};
static inline RedCtx make_ctx(const Partials &pt) { return RedCtx{pt.nblk, pt.part, pt.red, pt.stride}; }

// Loads issued where they stand: volatile inline PTX is neither sunk into the branch that uses it
// nor dropped, so a block's data is in flight while its control word (has this member converged?)
// and its CG scalar are still on their way.  nc: data the kernel does not write.
__device__ __forceinline__ float2 ld_early_nc(const float2 *p)
{
    float2 v;
    asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ double2 ld_early_nc(const double2 *p)
{
    double2 v;
    asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_early_nc(const float *p)
{
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double ld_early_nc(const double *p)
{
    double v;
    asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ unsigned int ld_early_nc_u32(const void *p)
{
    unsigned int v;
    asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ unsigned int ld_early_nc_u16(const void *p)
{
    unsigned short v;
    asm volatile("ld.global.nc.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}
// coherent variants for data the same thread writes back later in the kernel
__device__ __forceinline__ float2 ld_early(const float2 *p)
{
    float2 v;
    asm volatile("ld.global.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ double2 ld_early(const double2 *p)
{
    double2 v;
    asm volatile("ld.global.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
}

__device__ __forceinline__ double to_dbl(double v) { return v; }
__device__ __forceinline__ double to_dbl(float v) { return (double)v; }

// Publish a block partial of a per-member scalar; the blocks of one member are the kernel's
// blockIdx.x/y grid.  Returns true in the (single) last block to arrive, whose thread 0 then holds
// the fixed-order total in *total (sum, or max when is_max).  v is read in thread 0 only, where it
// is converted to double (a float, a double, or a df64 pair), so the other threads issue no FP64
// instruction for it.
template <class V>
__device__ __forceinline__ bool publish_partial(const RedCtx &rc, int slot, int m, V v, bool is_max, double *total)
{
    __shared__ bool s_last;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nb = gridDim.x * gridDim.y;
    double *p = rc.part + ((long long)slot * rc.stride + m) * rc.nblk;
    if (tid == 0) {
        p[blockIdx.x + blockIdx.y * gridDim.x] = to_dbl(v);
        __threadfence();
        unsigned int t = atomicAdd(&rc.red[m].cnt[slot], 1u);
        s_last = (t == (unsigned int)nb - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    if (tid < 32) {
        double acc = 0.0;
        for (int k = tid; k < nb; k += 32) {
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

template <class T> __device__ __forceinline__ const T *cw_of(const Level &L);
template <> __device__ __forceinline__ const float *cw_of<float>(const Level &L) { return L.cwf; }
template <> __device__ __forceinline__ const double *cw_of<double>(const Level &L) { return L.cwd; }
template <class T> __device__ __forceinline__ const T *cs_of(const Level &L);
template <> __device__ __forceinline__ const float *cs_of<float>(const Level &L) { return L.csf; }
template <> __device__ __forceinline__ const double *cs_of<double>(const Level &L) { return L.csd; }

static inline int cdiv(int a, int b) { return (a + b - 1) / b; }
static inline int round_up(int a, int b) { return cdiv(a, b) * b; }

// ------------------------------------------------------------- launch accounting
// Kernels launched directly on a stream (graph capture excluded; graph replays are counted by
// the C ABI from the captured graphs' kernel nodes).
void count_launches(long long n);
long long launches_so_far();
void set_capturing(bool on);
long long captured_launches();          // launches recorded into graphs by this thread so far
void note_capture_failure();            // a capture step failed: the graph must not be used
bool capture_failed();
unsigned long long conditional_body_launches();   // kernels run by conditional graph-node bodies

// ------------------------------------------------------------- launchers
// Flow kernels (k_flow.cu).  TR = tendency precision (float in mixed mode).
template <class TR>
void launch_predict(const Grid &g, int M, const double *u, const double *v, const double *p,
                    TR *Ru, TR *Rv, double *us, double *vs, const double *ubc, const double *frect,
                    const MemberCtl *ctl, cudaStream_t st);
void launch_reset(const Grid &g, int M, const double *u0, const double *v0, double *u, double *v, double *p,
                  double *x, void *Ru, void *Rv, size_t tend_bytes, double *wf, double *wd, int want_welford,
                  MemberCtl *ctl, cudaStream_t st);
void launch_outflow(const Grid &g, int M, const double *u, double *ubc, MemberCtl *ctl, cudaStream_t st);
void launch_rhs(const Grid &g, int M, const double *us, const double *vs, double *b, MemberCtl *ctl,
                cudaStream_t st);
void launch_recenter(const Grid &g, int M, double *x, const Partials &pt, long long nfluid, cudaStream_t st);
// Member 0's cell-centred velocity in the cost window, which the other members' Welford of
// d = u - u_0 needs (the exact contraction Y^T (Hq_0 - y) of the DOMAIN cost): batched runs read
// member 0's predictor and pressure increment (slot 0, unchanged during the correction); a
// one-member-at-a-time run stores member 0's samples in traj [n_window][2][S] and reads them back.
struct RefMember {
    const double *us, *vs, *x;      // FP64 batched: member 0's u*, v*, increment (nullptr otherwise)
    double *traj;                   // FP64 plain: member 0's window samples (nullptr otherwise)
};
void launch_correct(const Grid &g, double x0, double y0, int M, double *u, double *v, double *p,
                    const double *us, const double *vs, const double *x, double *wf, double *wd, RefMember ref,
                    int want_welford, double *series, const Partials &pt, MemberCtl *ctl, double div_tol,
                    long long nfluid, cudaStream_t st);
void launch_set_gidx(MemberCtl *ctl, int M, int base, cudaStream_t st);
void launch_copy_status(const MemberCtl *ctl, int M, int *status, cudaStream_t st);
void launch_load_ic(const Grid &g, const double *u0, const double *v0, double *u, double *v, cudaStream_t st);
// Window costs: J_domain = dx dy/(2 n_w) sum M2, J_sensor (two-pass over the series), and, when wd is
// given, Yd = dx dy/(2 n_w) sum M2_d = 1/2 ||h_m - h_0||^2 (the squared norm of eps Y_m).
void launch_cost(const Grid &g, int M, const double *wf, const double *wd, const double *series, double *J_domain,
                 double *J_sensor, double *Yd, double *part, cudaStream_t st);
void launch_export_state(const Grid &g, const double *u, const double *v, const double *p, double *uo,
                         double *vo, double *po, cudaStream_t st);

// Poisson kernels (k_poisson.cu).  TM = multigrid / inner-CG precision.
struct PoissonBufs {
    MixState ms;                    // mixed mode: df64 b and x live here
    double *b, *x;                  // level-0 FP64 right-hand side and solution (FP64 modes)
    void *r, *e, *z, *pv, *pv1, *q; // level-0 inner vectors (TM); pv, pv1: the two search directions
    void *lev_e[MAX_LEVELS];        // level >= 1 correction (TM)
    void *lev_f[MAX_LEVELS];        // level >= 1 right-hand side (TM)
    void *lev_t[MAX_LEVELS];        // pre-smoothed guess of each tiled level (level 0 included)
    int *refine_count;              // refinements done in the current step (one counter per member group)
};
struct PoissonCfg {
    int nlev;                       // number of levels
    int ncoarse;                    // first level handled by the per-member coarse kernel
    int nu_pre, nu_post, coarse_sweeps;
    int nu_c;                       // sweep pairs on the levels below the finest (0: nu_pre / nu_post)
    int max_outer, max_inner;
    double inner_rtol2;             // inner_rtol^2
    double rtol_abs;                // outer stop: max |r| <= rtol_abs (r = b - A x, FV form)
    int df_outer;                   // 1: outer residual / update in df64 (mixed mode)
    int conditional_loop;           // 1: refinement loop as a conditional WHILE graph node when captured
    MixConst mc;
    const unsigned char *cimg;      // coarse-block shared-memory image of the coarse levels' constants
    int cimg_bytes;                 // its size (a multiple of 16)
};
// Shared-memory layout of the coarse block (levels lc .. nlev-1).  The constant part (per level:
// west-face conductances [ny][nx+1], south-face conductances [ny+1][nx] in TM, fluid flags
// [ny][nx] bytes) comes first and is copied verbatim from an image built once; the per-level
// guess e [ny][nx] and right-hand side f [ny][nx] follow.  Offsets in bytes, each 16-aligned.
struct CoarseLayout {
    int cw[MAX_LEVELS], cs[MAX_LEVELS], fl[MAX_LEVELS], e[MAX_LEVELS];
    int image_bytes, total_bytes;
};
CoarseLayout coarse_layout(const Level *lev, int lc, int nlev, size_t tsz);
template <class TM> void prepare_poisson_kernels();
// The largest number of r^T z partials (blocks per member) a level-0 post-smoothing launch leaves (any sweep count).
int rz_parts_max(const Level &L0, bool mixed);
template <class TM>
void launch_vcycle(const Grid &g, const Level *lev, int M, const PoissonBufs &B, const PoissonCfg &pc,
                   const Partials &pt, MemberCtl *ctl, cudaStream_t st);
template <class TM>
void launch_cells_in(const Grid &g, const double *src, TM *dst, cudaStream_t st);
template <class TM>
void launch_cells_out(const Grid &g, const TM *src, double *dst, cudaStream_t st);
// Launch ONE kernel of the pressure solve (for standalone timing):
//   1 level-0 pre-smoothing + restriction, 2 level-0 prolongation + post-smoothing + dot,
//   3 inner SpMV, 4 inner AXPY, 5 outer FP64 residual, 7 coarse-level block kernel.
template <class TM>
int launch_poisson_single(int which, const Grid &g, const Level *lev, int M, const PoissonBufs &B,
                          const PoissonCfg &pc, const Partials &pt, MemberCtl *ctl, cudaStream_t st);
template <class TM>
void launch_pressure_solve(const Grid &g, const Level *lev, int M, const PoissonBufs &B, const PoissonCfg &pc,
                           const Partials &pt, MemberCtl *ctl, cudaStream_t st);

// Mixed-precision kernels (k_mixed.cu)
void launch_load_ic_mx(const Grid &g, const double *u0, const double *v0, const MixState &s0, cudaStream_t st);
void launch_reset_mx(const Grid &g, int M, const MixState &ic, const MixState &s, MemberCtl *ctl, int want_welford,
                     cudaStream_t st);
void launch_export_mx(const Grid &g, const MixState &s, long long off, double *uo, double *vo, double *po,
                      cudaStream_t st);
void launch_outflow_mx(const Grid &g, int M, const MixState &s, double *ubc, MemberCtl *ctl, cudaStream_t st);
// red, nfluid: the members' reductions (the fluid sum of the last increment) for the extrapolated
// initial guess of the pressure increment (s.xp set), none without it.
void launch_predict_rhs_mx(const Grid &g, const MixConst &K, int M, const MixState &s, const double *ubc,
                           const float *inh, const float *inl, const MemberCtl *ctl, const MemberRed *red,
                           long long nfluid, cudaStream_t st);
// The df64 residual leaves block partials; finish = 1 forms the totals and the convergence test
// right after it (k_res_finish), finish = 0 leaves them to the refinement loop's condition kernel
// (res_finish_member in res_finish.cuh).
void launch_outer_residual_mx(const Grid &g, const Level &L0, const MixConst &K, int M, const MixState &s, float *r,
                              float *e, const RedCtx &rc, MemberCtl *ctl, double rtol_abs, int count_it, int finish,
                              cudaStream_t st);
int outer_residual_parts_mx(const Grid &g);
// The last inner CG update fused with the refinement's x += e (df64 x).
void launch_axpy_last_mx(const Grid &g, int M, const MixState &s, const float *e, const float *p, const RedCtx &rc,
                         MemberCtl *ctl, int k, cudaStream_t st);
// ref: member 0's slot (its u*, v* and increment x are read for the Welford of d = u - u_0).
void launch_correct_mx(const Grid &g, const MixConst &K, int M, const MixState &s, const MixState &ref, double x0,
                       double y0, int want_welford, double *series, const Partials &pt, MemberCtl *ctl,
                       double div_tol, long long nfluid, cudaStream_t st);
// Per-member partial sums over fluid cells of a df64 plane pair (hi, lo) with member stride mstride.
void launch_plane_partial_mx(const Grid &g, int M, const float *hi, const float *lo, long long mstride, double *part,
                             int nparts, cudaStream_t st);
void launch_cost_final(const Grid &g, int M, const double *part, const double *part_d, int nparts,
                       const double *series, double *J_domain, double *J_sensor, double *Yd, cudaStream_t st);

// Ensemble kernels (k_ensemble.cu)
void launch_normals(unsigned long long seed, unsigned long long stream, long long first, long long n, double *out,
                    cudaStream_t st);
void launch_conv_sampler(int N, int nrx, int nry, int nxix, int nxiy, const double *Gx, const double *Gy,
                         const double *Z, const uint8_t *rect_ctrl, double sigma, double *Erect, double *tmp,
                         cudaStream_t st);
void launch_member_forcing(int M, int first_member, int N, int nrect, const double *Erect, const double *w,
                           double eps, double *frect, float *frect_f, cudaStream_t st);
void launch_rect_to_compact(int N, int nrect, int ncc, const int *cidx, const double *Erect, double *E,
                            cudaStream_t st);
void launch_compact_to_rect(int N, int nrect, int ncc, const int *cidx, const double *E, double *Erect,
                            cudaStream_t st);
// Gradients of Eq. (gradient_EnVar); a perturbed member whose status word is nonzero contributes no
// column of Y (its component keeps only the prior term (N-1) w_i).  status: N+1 ints (device).
void launch_sensor_gradient(int N, int n_window, const double *series, double eps, const double *w,
                            const int *status, double *g, cudaStream_t st);
void launch_scalar_gradient(int N, const double *J, const double *w, double eps, const int *status, double *g,
                            double *jprior, cudaStream_t st);
void launch_domain_gradient(int N, const double *J, const double *Yd, const double *w, double eps, const int *status,
                            double *g, cudaStream_t st);
void launch_df(int N, int n_ctrl, const double *E, const double *g, double scale, double *df, cudaStream_t st);
void launch_update_w(int N, double *w, const double *g, double step, cudaStream_t st);
void launch_d2f(long long n, const double *a, float *b, cudaStream_t st);
void launch_total_cost(const double *J, const double *jp, double *out, cudaStream_t st);

// Reduced-space optimisers (k_optim.cu)
void launch_sensor_anomalies(int N, int nw, const double *series, double eps, const int *status, double *mean,
                             double *Y, double *h0, cudaStream_t st);
void launch_gram(int N, long long nobs, const double *Y, const double *h0, const double *w, double *H, double *g,
                 cudaStream_t st);
void launch_cholesky_step(int N, const double *A, double *Lw, const double *g, const double *w, double alpha, double *x,
                          double *w_out, int *info, cudaStream_t st);
void launch_lbfgs_pair(int N, const double *w, const double *wp, const double *g, const double *gp, int slot,
                       double *S, double *Yh, double *sy, int m, cudaStream_t st);
void launch_lbfgs_direction(int N, int count, const int *order, const double *S, const double *Yh, const double *g,
                            double gamma0, double *q, double *alpha, double *p, double *gp, cudaStream_t st);
void launch_trial_point(int N, const double *w, const double *p, double a, double *wt, double *prior, cudaStream_t st);
void launch_h1_cg(int n, const int *nb, double dx, double dy, double l_sob, const double *g, double *x, double *work,
                  double rtol, int max_it, int *iters, cudaStream_t st);
void launch_scale_vec(long long n, double a, const double *x, double *y, cudaStream_t st);
void launch_axpy_vec(long long n, double a, const double *x, double *y, cudaStream_t st);
void launch_dot_max(long long n, const double *a, const double *b, double *out, cudaStream_t st);

// Eigenvector ensemble (k_eigen.cu)
size_t eigen_work_doubles(int nrx, int nry, int ncc, int mmax, int k);
int eigen_ensemble(int nrx, int nry, double dx, double dy, double a, double sigma, int ncc, const int *cidx, int N,
                   int y_only, int m0, int mmax, double tol, unsigned long long seed, double *work, double *E,
                   double *lam_host, int *steps_host, double *bound_host, cudaStream_t st);

} // namespace envar
