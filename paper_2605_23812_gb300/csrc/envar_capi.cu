// envar_capi.cu -- the C ABI (include/envar.h): handle lifecycle, geometry and multigrid set-up,
// device buffers, CUDA-graph capture of the time step, and the EnVar calls of Fig. (envar_loop).
//
// Set-up (once per handle, host C++): cell mask of the open cavity, face kinds, inlet table,
// multigrid hierarchy (masks and face conductances), control rectangle.  Everything per
// iteration -- ensemble draws, forcings, the N+1 forward runs, costs, gradient and update -- runs
// in the library's CUDA kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "envar_internal.cuh"
#include "revolve.h"
#include "../../include/envar.h"

namespace envar {
void launch_axis_factor(double h, double a, int ncell, int m, int pad, int nxi, double *G, cudaStream_t st);
}
using namespace envar;

constexpr int ENVAR_MAX_GROUPS = 8;

// Limited-memory BFGS history in device memory (Sec. 3.3.1, Eq. update_BFGS): the newest `count`
// of at most m pairs (s, y) in ring slots, with the previous iterate and gradient.
struct LbfgsState {
    int n = 0, m = 0, count = 0, head = 0;
    bool have_prev = false;
    double *S = nullptr, *Y = nullptr, *sy = nullptr, *q = nullptr, *a = nullptr, *p = nullptr, *gp = nullptr;
    double *xprev = nullptr, *gprev = nullptr;
    int *order = nullptr;
};

struct GraphSet {
    cudaGraphExec_t many = nullptr;   // steps_per_graph steps
    cudaGraphExec_t one = nullptr;    // one step
    long long kernels_many = 0, kernels_one = 0;   // kernel nodes per replay
};
static std::atomic<long long> g_graph_kernels{0};

struct envar_handle_s {
    envar_config cfg{};
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int N = 0, Mall = 0;              // perturbations, member slots
    bool batched = true, mixed = false;
    Grid g{};
    double x0 = 0, y0 = 0;
    long long nfluid = 0;
    // levels
    int nlev = 0, ncoarse = 0;
    Level lev[MAX_LEVELS]{};
    // control
    int ia = 0, ja = 0, nrx = 0, nry = 0, ncc = 0, n_ctrl = 0, nrect = 0;
    int *d_cidx = nullptr;
    uint8_t *d_rect_ctrl = nullptr;
    double *d_Erect = nullptr, *d_E = nullptr, *d_frect = nullptr;
    // state
    double *d_u0 = nullptr, *d_v0 = nullptr;
    double *d_u = nullptr, *d_v = nullptr, *d_us = nullptr, *d_vs = nullptr, *d_p = nullptr;
    void *d_Ru = nullptr, *d_Rv = nullptr;
    size_t tend_bytes = 0;
    double *d_ubc = nullptr, *d_wf = nullptr, *d_series_slot = nullptr, *d_series = nullptr;
    double *d_wd = nullptr;           // FP64 Welford of d = u - u_0 (3 planes per member slot)
    double *d_traj = nullptr;         // FP64_PLAIN: member 0's window samples [n_window][2][S]
    int *d_status = nullptr;          // status words of the N+1 members of the last forward run
    PoissonBufs pb{};
    PoissonCfg pc{};
    Partials pt{};
    MemberCtl *d_ctl = nullptr;
    // mixed-precision state (ENVAR_MIXED)
    MixState ms{}, ic{};
    MixConst mc{};
    float *d_inh = nullptr, *d_inl = nullptr;
    // results
    double *d_Jd_slot = nullptr, *d_Js_slot = nullptr, *d_Jd = nullptr, *d_Js = nullptr, *d_costpart = nullptr;
    double *d_Yd_slot = nullptr, *d_Yd = nullptr;   // 1/2 ||h_m - h_0||^2 per member (DOMAIN)
    double *d_w = nullptr, *d_g = nullptr, *d_jprior = nullptr, *d_gscalar = nullptr;
    std::vector<MemberCtl> ctl_all;
    bool have_forward = false, have_ic = false;
    int last_member_slot0 = -1;       // member held in slot 0 after a plain-mode run
    std::vector<void *> allocs;
    GraphSet graphs[2];               // [0]: all slots, [1]: one slot
    // discrete adjoint (FP64 handles): work planes, checkpoint slots, reverse-step graphs
    double *d_adj = nullptr;
    double *d_snap = nullptr;
    int n_snap = 0;
    cudaGraphExec_t adj_graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [first step][in window]
    long long adj_fwd_steps = 0, adj_rev_steps = 0, adj_stores = 0, adj_restores = 0;
    unsigned char *d_flush = nullptr;   // L2 eviction buffer of envar_time_kernel
    unsigned char *d_cimg = nullptr;    // coarse-block constants image
    int ngroups = 1;                    // concurrent member groups of the captured step
    cudaStream_t side[ENVAR_MAX_GROUPS] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[ENVAR_MAX_GROUPS] = {};
    cudaEvent_t ev_solved0 = nullptr;   // member 0's pressure increment is final (group 0)
    cudaEvent_t ev_corr[ENVAR_MAX_GROUPS] = {};   // a group's correction has read member 0's increment
    int cimg_bytes = 0;
    // reduced-space optimisers (allocated on first use)
    double *d_Y = nullptr, *d_h0 = nullptr, *d_smean = nullptr, *d_H = nullptr, *d_L = nullptr, *d_x = nullptr;
    int *d_info = nullptr;
    double *d_wt = nullptr, *d_prior_t = nullptr;
    LbfgsState lbw, lbf;                // L-BFGS histories: ensemble weights w, control vector f
    int *d_cnb = nullptr;               // control-cell neighbours E, W, N, S (-1: none) [4][n_cc]
    double *d_h1 = nullptr;             // H^1 smoothing work (3 n_cc) and adjoint-loop vectors
    double *d_fg = nullptr, *d_fgs = nullptr, *d_fs = nullptr, *d_dm = nullptr;
    int *d_h1it = nullptr;
    char err[512] = {0};
};

static char g_init_err[512];
namespace envar {
void set_global_error(const char *msg) { std::snprintf(g_init_err, sizeof(g_init_err), "%s", msg); }
}

static void set_err(envar_handle h, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h ? h->err : g_init_err, sizeof(g_init_err), fmt, ap);
    va_end(ap);
}

#define CK(call)                                                                             \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            set_err(h, "%s failed: %s", #call, cudaGetErrorString(e_));                      \
            return ENVAR_ECUDA;                                                              \
        }                                                                                    \
    } while (0)

template <class T>
static int dalloc(envar_handle h, T **p, size_t count)
{
    void *q = nullptr;
    size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        set_err(h, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
        *p = nullptr;
        return ENVAR_ENOMEM;
    }
    h->allocs.push_back(q);
    *p = reinterpret_cast<T *>(q);
    return ENVAR_OK;
}
#define DA(ptr, n)                                      \
    do {                                                \
        int rc_ = dalloc(h, &(ptr), (size_t)(n));       \
        if (rc_) return rc_;                            \
    } while (0)

extern "C" int envar_default_config(envar_config *c, int nx, int ny)
{
    if (!c) return ENVAR_EINVAL;
    std::memset(c, 0, sizeof(*c));
    c->nx = nx; c->ny = ny;
    c->x0 = -1.2; c->x1 = 2.5; c->y0 = -1.0; c->y1 = 1.0;
    c->Re = 1000.0; c->cfl = 0.3; c->inlet_delta = 0.1; c->conv_speed = 1.0;
    c->n_steps = 1000; c->n_window = 500; c->n_members = 8;
    c->region[0] = -0.5; c->region[1] = 1.0; c->region[2] = -0.2; c->region[3] = 0.3;
    c->sigma = 0.1; c->corr_len = 0.05; c->eps = 1e-2; c->seed = 1000ULL;
    c->precision = ENVAR_MIXED; c->cost_mode = ENVAR_COST_DOMAIN;
    c->div_tol = 1e-10; c->max_outer = 4; c->max_inner = 6; c->inner_rtol = 1e-4;
    c->nu_pre = 2; c->nu_post = 2; c->coarse_sweeps = 8; c->steps_per_graph = 10;
    c->lip_slip = 0; c->noslip_span[0] = -0.4; c->noslip_span[1] = 1.75; c->forcing_y_only = 0;
    c->conditional_refinement = 1;
    c->guess_extrapolation = 1;
    c->nu_coarse = 0;
    return ENVAR_OK;
}

// ------------------------------------------------------------------------------------ set-up
static int build_geometry(envar_handle h)
{
    const envar_config &c = h->cfg;
    const int nx = c.nx, ny = c.ny;
    const double dx = (c.x1 - c.x0) / nx, dy = (c.y1 - c.y0) / ny;
    const int P = round_up(nx + 1, 32);
    const long long S = (long long)(ny + 1) * P;
    Grid &g = h->g;
    g.nx = nx; g.ny = ny; g.P = P; g.S = S;
    g.dx = dx; g.dy = dy; g.dt = c.cfl * std::min(dx, dy); g.nu = 1.0 / c.Re;
    g.cx = dy / dx; g.cy = dx / dy; g.hxy = dx * dy;
    g.n_steps = c.n_steps; g.n_window = c.n_window; g.conv_speed = c.conv_speed;
    h->x0 = c.x0; h->y0 = c.y0;

    auto xc = [&](int i) { return c.x0 + ((double)i + 0.5) * dx; };
    auto yc = [&](int j) { return c.y0 + ((double)j + 0.5) * dy; };
    std::vector<uint8_t> F((size_t)S, 0), uk((size_t)S, FK_ZERO), vk((size_t)S, FK_ZERO);
    long long nfl = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double x = xc(i), y = yc(j);
            bool f = (y > 0.0) || (x > 0.0 && x < 1.0);
            F[(size_t)j * P + i] = f;
            nfl += f;
        }
    h->nfluid = nfl;
    auto fl = [&](int i, int j) -> int {
        if (i < 0 || i >= nx || j < 0 || j >= ny) return 0;
        return F[(size_t)j * P + i];
    };
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            uint8_t k;
            if (i == 0) k = fl(0, j) ? FK_INLET : FK_ZERO;
            else if (i == nx) k = fl(nx - 1, j) ? FK_OUTLET : FK_ZERO;
            else {
                int a = fl(i - 1, j), b = fl(i, j);
                k = (a && b) ? FK_UNK : ((a || b) ? FK_ZERO : FK_SOLID);
            }
            uk[(size_t)j * P + i] = k;
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            uint8_t k;
            if (j == 0 || j == ny) k = FK_ZERO;
            else {
                int a = fl(i, j - 1), b = fl(i, j);
                k = (a && b) ? FK_UNK : ((a || b) ? FK_ZERO : FK_SOLID);
            }
            vk[(size_t)j * P + i] = k;
        }
    // slip segments of the lower wall: a solid face under a fluid face reflects evenly
    if (c.lip_slip)
        for (int j = 0; j + 1 < ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                const double xf = c.x0 + (double)i * dx;
                if (uk[(size_t)j * P + i] == FK_SOLID && uk[(size_t)(j + 1) * P + i] == FK_UNK &&
                    (xf < c.noslip_span[0] || xf > c.noslip_span[1]))
                    uk[(size_t)j * P + i] = FK_SLIP;
            }
    // the mirror rule needs a solid layer at least two faces thick
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i)
            if (uk[(size_t)j * P + i] == FK_SOLID && j > 0 && j + 1 < ny && uk[(size_t)(j - 1) * P + i] == FK_UNK &&
                uk[(size_t)(j + 1) * P + i] == FK_UNK) {
                set_err(h, "geometry: one-cell-thick solid layer is not supported");
                return ENVAR_EINVAL;
            }
    std::vector<double> uin((size_t)ny, 0.0);
    for (int j = 0; j < ny; ++j)
        if (uk[(size_t)j * P] == FK_INLET) uin[j] = std::erf(yc(j) / c.inlet_delta);

    uint8_t *dF, *duk, *dvk;
    double *duin;
    DA(dF, S); DA(duk, S); DA(dvk, S); DA(duin, ny);
    CK(cudaMemcpy(dF, F.data(), S, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(duk, uk.data(), S, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dvk, vk.data(), S, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(duin, uin.data(), sizeof(double) * ny, cudaMemcpyHostToDevice));
    g.fluid = dF; g.uk = duk; g.vk = dvk; g.u_in = duin;
    {
        std::vector<float> ih((size_t)ny), il((size_t)ny);
        for (int j = 0; j < ny; ++j) {
            ih[j] = (float)uin[j];
            il[j] = (float)(uin[j] - (double)ih[j]);
        }
        DA(h->d_inh, ny); DA(h->d_inl, ny);
        CK(cudaMemcpy(h->d_inh, ih.data(), sizeof(float) * ny, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->d_inl, il.data(), sizeof(float) * ny, cudaMemcpyHostToDevice));
    }

    // ---- multigrid hierarchy
    struct HostLevel { int nx, ny, P; long long S; std::vector<uint8_t> F; std::vector<double> cw, cs; };
    std::vector<HostLevel> hl;
    {
        HostLevel L0{nx, ny, P, S, F, std::vector<double>((size_t)S, 0.0), std::vector<double>((size_t)S, 0.0)};
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx; ++i)
                if (uk[(size_t)j * P + i] == FK_UNK) L0.cw[(size_t)j * P + i] = g.cx;
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i < nx; ++i)
                if (vk[(size_t)j * P + i] == FK_UNK) L0.cs[(size_t)j * P + i] = g.cy;
        hl.push_back(std::move(L0));
    }
    while ((int)hl.size() < MAX_LEVELS) {
        const HostLevel &f = hl.back();
        if (f.nx % 2 || f.ny % 2 || f.nx / 2 < 4 || f.ny / 2 < 2) break;
        HostLevel cL;
        cL.nx = f.nx / 2; cL.ny = f.ny / 2; cL.P = round_up(cL.nx + 1, 32); cL.S = (long long)(cL.ny + 1) * cL.P;
        cL.F.assign((size_t)cL.S, 0); cL.cw.assign((size_t)cL.S, 0.0); cL.cs.assign((size_t)cL.S, 0.0);
        for (int J = 0; J < cL.ny; ++J)
            for (int I = 0; I < cL.nx; ++I) {
                int any = 0;
                for (int dj = 0; dj < 2; ++dj)
                    for (int di = 0; di < 2; ++di) any |= f.F[(size_t)(2 * J + dj) * f.P + 2 * I + di];
                cL.F[(size_t)J * cL.P + I] = (uint8_t)any;
            }
        for (int J = 0; J < cL.ny; ++J)
            for (int I = 0; I <= cL.nx; ++I)
                cL.cw[(size_t)J * cL.P + I] =
                    0.5 * (f.cw[(size_t)(2 * J) * f.P + 2 * I] + f.cw[(size_t)(2 * J + 1) * f.P + 2 * I]);
        for (int J = 0; J <= cL.ny; ++J)
            for (int I = 0; I < cL.nx; ++I)
                cL.cs[(size_t)J * cL.P + I] =
                    0.5 * (f.cs[(size_t)(2 * J) * f.P + 2 * I] + f.cs[(size_t)(2 * J) * f.P + 2 * I + 1]);
        hl.push_back(std::move(cL));
    }
    h->nlev = (int)hl.size();
    if (h->nlev < 2) {
        set_err(h, "grid %dx%d too small for the multigrid hierarchy", nx, ny);
        return ENVAR_EINVAL;
    }
    // the coarse block starts at the first level from which all levels fit its shared memory
    const size_t tsz = h->mixed ? sizeof(float) : sizeof(double);
    Level dims[MAX_LEVELS]{};
    for (int l = 0; l < h->nlev; ++l) { dims[l].nx = hl[l].nx; dims[l].ny = hl[l].ny; }
    auto coarse_bytes = [&](int lc) { return (size_t)coarse_layout(dims, lc, h->nlev, tsz).total_bytes; };
    h->ncoarse = h->nlev - 1;
    for (int l = 1; l < h->nlev; ++l)
        if (coarse_bytes(l) <= (size_t)COARSE_SMEM_MAX) { h->ncoarse = l; break; }
    for (int l = 0; l < h->nlev; ++l) {
        const HostLevel &L = hl[l];
        uint8_t *dfl;
        float *cwf, *csf;
        double *cwd, *csd;
        if (l == 0) dfl = dF; else { DA(dfl, L.S); CK(cudaMemcpy(dfl, L.F.data(), L.S, cudaMemcpyHostToDevice)); }
        std::vector<float> f1(L.cw.begin(), L.cw.end()), f2(L.cs.begin(), L.cs.end());
        DA(cwf, L.S); DA(csf, L.S); DA(cwd, L.S); DA(csd, L.S);
        CK(cudaMemcpy(cwf, f1.data(), sizeof(float) * L.S, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(csf, f2.data(), sizeof(float) * L.S, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(cwd, L.cw.data(), sizeof(double) * L.S, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(csd, L.cs.data(), sizeof(double) * L.S, cudaMemcpyHostToDevice));
        h->lev[l] = Level{L.nx, L.ny, L.P, L.S, dfl, cwf, csf, cwd, csd, nullptr, 0.0, 0.0, 0.f, 0.f, nullptr, nullptr, nullptr};
        if (l == 0 || L.nx % 2) continue;   // the coded smoother works on cell pairs
        // conductance codes: the distinct conductances of each direction in first-seen order
        std::vector<double> tx, ty;
        auto index_of = [](std::vector<double> &t, double v) -> int {
            for (size_t k = 0; k < t.size(); ++k)
                if (t[k] == v) return (int)k;
            t.push_back(v);
            return (int)t.size() - 1;
        };
        std::vector<uint16_t> code((size_t)L.S, 0);
        bool fits = true;
        for (int j = 0; j < L.ny && fits; ++j)
            for (int i = 0; i < L.nx && fits; ++i) {
                const size_t c = (size_t)j * L.P + i;
                const int kw = index_of(tx, L.cw[c]), ke = index_of(tx, L.cw[c + 1]);
                const int ks = index_of(ty, L.cs[c]), kn = index_of(ty, L.cs[c + L.P]);
                if (tx.size() > 16 || ty.size() > 16) { fits = false; break; }
                code[c] = (uint16_t)(kw | (ke << 4) | (ks << 8) | (kn << 12));
            }
        if (!fits) continue;   // this level keeps the explicit-conductance smoother
        std::vector<double> td(32, 0.0);
        std::vector<float> tf(32, 0.f);
        for (size_t k = 0; k < tx.size(); ++k) { td[k] = tx[k]; tf[k] = (float)tx[k]; }
        for (size_t k = 0; k < ty.size(); ++k) { td[16 + k] = ty[k]; tf[16 + k] = (float)ty[k]; }
        uint16_t *dcode;
        float *dtf;
        double *dtd;
        DA(dcode, L.S); DA(dtf, 32); DA(dtd, 32);
        CK(cudaMemcpy(dcode, code.data(), sizeof(uint16_t) * L.S, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dtf, tf.data(), sizeof(float) * 32, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dtd, td.data(), sizeof(double) * 32, cudaMemcpyHostToDevice));
        h->lev[l].code = dcode;
        h->lev[l].ktabf = dtf;
        h->lev[l].ktabd = dtd;
    }
    {   // constant part of the coarse block's shared memory (conductances and fluid flags)
        const CoarseLayout lay = coarse_layout(dims, h->ncoarse, h->nlev, tsz);
        std::vector<unsigned char> im((size_t)lay.image_bytes, 0);
        auto put = [&](int byte_off, size_t idx, double v) {
            if (h->mixed) { const float f = (float)v; std::memcpy(&im[byte_off + 4 * idx], &f, 4); }
            else std::memcpy(&im[byte_off + 8 * idx], &v, 8);
        };
        for (int l = h->ncoarse; l < h->nlev; ++l) {
            const HostLevel &L = hl[l];
            for (int j = 0; j < L.ny; ++j)
                for (int i = 0; i <= L.nx; ++i) put(lay.cw[l], (size_t)j * (L.nx + 1) + i, L.cw[(size_t)j * L.P + i]);
            for (int j = 0; j <= L.ny; ++j)
                for (int i = 0; i < L.nx; ++i) put(lay.cs[l], (size_t)j * L.nx + i, L.cs[(size_t)j * L.P + i]);
            for (int j = 0; j < L.ny; ++j)
                for (int i = 0; i < L.nx; ++i) im[lay.fl[l] + (size_t)j * L.nx + i] = L.F[(size_t)j * L.P + i];
        }
        DA(h->d_cimg, im.size());
        CK(cudaMemcpy(h->d_cimg, im.data(), im.size(), cudaMemcpyHostToDevice));
        h->cimg_bytes = lay.image_bytes;
    }
    {   // level-0 open-face bits (W 1, E 2, S 4, N 8) of fluid cells
        std::vector<uint8_t> op((size_t)S, 0);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                if (!F[(size_t)j * P + i]) continue;
                uint8_t b = 0;
                b |= (uk[(size_t)j * P + i] == FK_UNK) ? 1 : 0;
                b |= (uk[(size_t)j * P + i + 1] == FK_UNK) ? 2 : 0;
                b |= (vk[(size_t)j * P + i] == FK_UNK) ? 4 : 0;
                b |= (vk[(size_t)(j + 1) * P + i] == FK_UNK) ? 8 : 0;
                op[(size_t)j * P + i] = b;
            }
        uint8_t *dop;
        DA(dop, S);
        CK(cudaMemcpy(dop, op.data(), S, cudaMemcpyHostToDevice));
        h->lev[0].open = dop;
        h->lev[0].cx = g.cx;
        h->lev[0].cy = g.cy;
        h->lev[0].cxf = (float)g.cx;
        h->lev[0].cyf = (float)g.cy;
    }
    // coarse block must fit in shared memory
    if (coarse_bytes(h->ncoarse) > (size_t)COARSE_SMEM_MAX) {
        set_err(h, "coarse multigrid levels (%zu bytes) exceed shared memory; use nx, ny with more factors of 2",
                coarse_bytes(h->ncoarse));
        return ENVAR_EINVAL;
    }

    // ---- control rectangle (Sec. 4.1): cells with centre inside the region, inclusive
    int ia = -1, ib = -1, ja = -1, jb = -1;
    for (int i = 0; i < nx; ++i) {
        double x = xc(i);
        if (x >= c.region[0] && x <= c.region[1]) { if (ia < 0) ia = i; ib = i; }
    }
    for (int j = 0; j < ny; ++j) {
        double y = yc(j);
        if (y >= c.region[2] && y <= c.region[3]) { if (ja < 0) ja = j; jb = j; }
    }
    if (ia < 0 || ja < 0) {
        set_err(h, "control region contains no cell centre");
        return ENVAR_EINVAL;
    }
    h->ia = ia; h->ja = ja; h->nrx = ib - ia + 1; h->nry = jb - ja + 1; h->nrect = h->nrx * h->nry;
    g.ia = ia; g.ja = ja; g.nrx = h->nrx; g.nry = h->nry;
    std::vector<int> cidx;
    std::vector<uint8_t> rc((size_t)h->nrect, 0);
    for (int j = ja; j <= jb; ++j)
        for (int i = ia; i <= ib; ++i)
            if (F[(size_t)j * P + i]) {
                int r = (j - ja) * h->nrx + (i - ia);
                cidx.push_back(r);
                rc[r] = 1;
            }
    h->ncc = (int)cidx.size();
    h->n_ctrl = 2 * h->ncc;
    {   // control-cell neighbours (E, W, N, S) inside the control set, for the H^1 smoothing
        std::vector<int> where((size_t)h->nrect, -1), nb((size_t)4 * std::max(h->ncc, 1), -1);
        for (int q = 0; q < h->ncc; ++q) where[cidx[q]] = q;
        for (int q = 0; q < h->ncc; ++q) {
            const int r = cidx[q], a = r % h->nrx, b = r / h->nrx;
            if (a + 1 < h->nrx) nb[q] = where[r + 1];
            if (a > 0) nb[(size_t)h->ncc + q] = where[r - 1];
            if (b + 1 < h->nry) nb[2 * (size_t)h->ncc + q] = where[r + h->nrx];
            if (b > 0) nb[3 * (size_t)h->ncc + q] = where[r - h->nrx];
        }
        DA(h->d_cnb, nb.size());
        CK(cudaMemcpy(h->d_cnb, nb.data(), sizeof(int) * nb.size(), cudaMemcpyHostToDevice));
    }
    DA(h->d_cidx, std::max(h->ncc, 1));
    DA(h->d_rect_ctrl, h->nrect);
    CK(cudaMemcpy(h->d_cidx, cidx.data(), sizeof(int) * h->ncc, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_rect_ctrl, rc.data(), h->nrect, cudaMemcpyHostToDevice));
    return ENVAR_OK;
}

// Ensemble draw (Sec. 3.3.2): Z from Philox normals, then sigma (Gx (x) Gy) Z on the control cells.
static void sampler_axis(double hh, double a, int ncell, int *m, int *pad, int *nxi)
{
    int mm = (int)std::ceil(4.0 * hh / a);
    if (mm < 1) mm = 1;
    double eta = hh / mm;
    *m = mm;
    *pad = (int)std::ceil(5.0 * a / eta);
    *nxi = (ncell - 1) * mm + 1 + 2 * (*pad);
}

static int generate_ensemble(envar_handle h)
{
    const int N = h->N;
    if (N == 0) return ENVAR_OK;
    const double a = h->cfg.corr_len;
    int mx, px, nxix, my, py, nxiy;
    sampler_axis(h->g.dx, a, h->nrx, &mx, &px, &nxix);
    sampler_axis(h->g.dy, a, h->nry, &my, &py, &nxiy);
    double *Gx, *Gy, *Z, *T;
    size_t nz = (size_t)N * 2 * nxiy * nxix;
    if (cudaMalloc(&Gx, sizeof(double) * (size_t)h->nrx * nxix) != cudaSuccess ||
        cudaMalloc(&Gy, sizeof(double) * (size_t)h->nry * nxiy) != cudaSuccess ||
        cudaMalloc(&Z, sizeof(double) * nz) != cudaSuccess ||
        cudaMalloc(&T, sizeof(double) * (size_t)N * 2 * nxiy * h->nrx) != cudaSuccess) {
        set_err(h, "out of device memory while drawing the ensemble");
        return ENVAR_ENOMEM;
    }
    launch_axis_factor(h->g.dx, a, h->nrx, mx, px, nxix, Gx, h->st);
    launch_axis_factor(h->g.dy, a, h->nry, my, py, nxiy, Gy, h->st);
    launch_normals(h->cfg.seed, 0ULL, 0LL, (long long)nz, Z, h->st);
    launch_conv_sampler(N, h->nrx, h->nry, nxix, nxiy, Gx, Gy, Z, h->d_rect_ctrl, h->cfg.sigma, h->d_Erect, T, h->st);
    launch_rect_to_compact(N, h->nrect, h->ncc, h->d_cidx, h->d_Erect, h->d_E, h->st);
    if (h->cfg.forcing_y_only) {   // zero prior variance on the fx entries
        CK(cudaMemset2DAsync(h->d_E, sizeof(double) * h->n_ctrl, 0, sizeof(double) * h->ncc, N, h->st));
        launch_compact_to_rect(N, h->nrect, h->ncc, h->d_cidx, h->d_E, h->d_Erect, h->st);
    }
    CK(cudaStreamSynchronize(h->st));
    cudaFree(Gx); cudaFree(Gy); cudaFree(Z); cudaFree(T);
    CK(cudaGetLastError());
    return ENVAR_OK;
}

static int alloc_buffers(envar_handle h)
{
    const int M = h->Mall;
    const long long S = h->g.S;
    const size_t n0 = (size_t)S * M;
    const size_t tsz = h->mixed ? sizeof(float) : sizeof(double);
    if (h->mixed) {
        MixState &ms = h->ms;
        DA(ms.uh, n0); DA(ms.ul, n0); DA(ms.vh, n0); DA(ms.vl, n0);
        DA(ms.ush, n0); DA(ms.usl, n0); DA(ms.vsh, n0); DA(ms.vsl, n0);
        DA(ms.p, n0); DA(ms.Ru, 2 * n0); DA(ms.Rv, 2 * n0);
        ms.rstride = (long long)n0;
        DA(ms.bh, n0); DA(ms.bl, n0); DA(ms.xh, n0); DA(ms.xl, n0);
        if (h->cfg.guess_extrapolation) DA(ms.xp, n0);
        if (h->cfg.cost_mode == ENVAR_COST_DOMAIN) DA(ms.wf, 6 * n0);
        if (h->cfg.cost_mode == ENVAR_COST_DOMAIN && h->N > 0) DA(ms.wd, 4 * n0);
        DA(ms.frect, (size_t)M * 2 * h->nrect);
        DA(h->ic.uh, S); DA(h->ic.ul, S); DA(h->ic.vh, S); DA(h->ic.vl, S);
        CK(cudaMemset(h->ic.uh, 0, sizeof(float) * S)); CK(cudaMemset(h->ic.ul, 0, sizeof(float) * S));
        CK(cudaMemset(h->ic.vh, 0, sizeof(float) * S)); CK(cudaMemset(h->ic.vl, 0, sizeof(float) * S));
        h->pb.ms = ms;
    } else {
        DA(h->d_u0, S); DA(h->d_v0, S);
        DA(h->d_u, n0); DA(h->d_v, n0); DA(h->d_us, n0); DA(h->d_vs, n0); DA(h->d_p, n0);
        DA(h->pb.x, n0); DA(h->pb.b, n0);
        h->tend_bytes = tsz * n0;
        char *a, *b;
        DA(a, h->tend_bytes); DA(b, h->tend_bytes);
        h->d_Ru = a; h->d_Rv = b;
        if (h->cfg.cost_mode == ENVAR_COST_DOMAIN) DA(h->d_wf, 3 * n0);
        if (h->cfg.cost_mode == ENVAR_COST_DOMAIN && h->N > 0) {
            DA(h->d_wd, 3 * n0);
            if (!h->batched && h->cfg.n_window > 0) DA(h->d_traj, (size_t)h->cfg.n_window * 2 * S);
        }
    }
    DA(h->d_ubc, (size_t)M * h->g.ny);
    const int nw = std::max(h->cfg.n_window, 1);
    DA(h->d_series_slot, (size_t)M * nw * 8);
    h->d_series = h->d_series_slot;
    if (!h->batched) DA(h->d_series, (size_t)(h->N + 1) * nw * 8);
    // Poisson (TM)
    {
        char *r, *e, *z, *q, *pv;
        DA(r, tsz * n0); DA(e, tsz * n0); DA(z, tsz * n0); DA(q, tsz * n0); DA(pv, 2 * tsz * n0);
        h->pb.r = r; h->pb.e = e; h->pb.z = z; h->pb.q = q; h->pb.pv = pv; h->pb.pv1 = pv + tsz * n0;
        for (int l = 1; l < h->nlev; ++l) {
            char *le, *lf;
            DA(le, tsz * (size_t)h->lev[l].S * M); DA(lf, tsz * (size_t)h->lev[l].S * M);
            h->pb.lev_e[l] = le; h->pb.lev_f[l] = lf;
        }
        for (int l = 0; l < h->ncoarse; ++l) {
            char *lt;
            DA(lt, tsz * (size_t)h->lev[l].S * M);
            h->pb.lev_t[l] = lt;
        }
    }
    // capacity for every partial-producing tiling (per-block partials)
    h->pt.nblk = std::max(cdiv(h->g.nx, 32) * cdiv(h->g.ny, 16), rz_parts_max(h->lev[0], h->mixed));
    h->pt.stride = M;
    DA(h->pt.part, (size_t)RS_COUNT * M * h->pt.nblk);
    DA(h->pt.red, M);
    DA(h->pb.refine_count, M);
    CK(cudaMemset(h->pb.refine_count, 0, sizeof(int) * M));
    CK(cudaMemset(h->pt.red, 0, sizeof(MemberRed) * M));
    DA(h->d_ctl, M);
    CK(cudaMemset(h->d_ctl, 0, sizeof(MemberCtl) * M));
    // ensemble / results
    const int N = h->N;
    DA(h->d_Erect, (size_t)std::max(N, 1) * 2 * h->nrect);
    DA(h->d_E, (size_t)std::max(N, 1) * h->n_ctrl);
    DA(h->d_frect, (size_t)M * 2 * h->nrect);
    DA(h->d_Jd_slot, M); DA(h->d_Js_slot, M);
    DA(h->d_Jd, N + 1); DA(h->d_Js, N + 1);
    DA(h->d_costpart, (size_t)2 * 64 * M);
    DA(h->d_Yd_slot, M); DA(h->d_Yd, N + 1);
    CK(cudaMemset(h->d_Yd, 0, sizeof(double) * (N + 1)));
    DA(h->d_status, N + 1);
    CK(cudaMemset(h->d_status, 0, sizeof(int) * (N + 1)));
    DA(h->d_w, std::max(N, 1)); DA(h->d_g, std::max(N, 1)); DA(h->d_jprior, 1); DA(h->d_gscalar, std::max(N, 1));
    DA(h->d_wt, std::max(N, 1));
    CK(cudaMemset(h->d_w, 0, sizeof(double) * std::max(N, 1)));
    return ENVAR_OK;
}

// ------------------------------------------------------------------------------------ stepping
// The per-member arrays of member slots m0, m0+1, ...: every such array is laid out member-major,
// so a group of members is a pointer offset (the partials keep the handle's member stride).
struct MemberView {
    MixState ms;
    PoissonBufs pb;
    Partials pt;
    MemberCtl *ctl;
    double *ubc, *series, *u, *v, *us, *vs, *p, *wf, *wd, *frect;
    void *Ru, *Rv;
};
static MemberView member_view(envar_handle h, int m0)
{
    const long long S = h->g.S, o = (long long)m0 * S;
    const size_t tsz = h->mixed ? sizeof(float) : sizeof(double);
    auto fs = [&](float *q, long long k) { return q ? q + k : q; };
    auto ds = [&](double *q, long long k) { return q ? q + k : q; };
    auto vs = [&](void *q, long long elems) { return q ? (void *)((char *)q + tsz * elems) : q; };
    MemberView v;
    v.ms = h->ms;
    if (h->mixed) {
        MixState &w = v.ms;
        w.uh = fs(w.uh, o); w.ul = fs(w.ul, o); w.vh = fs(w.vh, o); w.vl = fs(w.vl, o);
        w.ush = fs(w.ush, o); w.usl = fs(w.usl, o); w.vsh = fs(w.vsh, o); w.vsl = fs(w.vsl, o);
        w.p = fs(w.p, o); w.Ru = fs(w.Ru, o); w.Rv = fs(w.Rv, o);
        w.bh = fs(w.bh, o); w.bl = fs(w.bl, o); w.xh = fs(w.xh, o); w.xl = fs(w.xl, o);
        w.xp = fs(w.xp, o);
        w.wf = fs(w.wf, 6 * o);
        w.wd = fs(w.wd, 4 * o);
        w.frect = fs(w.frect, (long long)m0 * 2 * h->nrect);
    }
    v.pb = h->pb;
    v.pb.ms = v.ms;
    v.pb.b = ds(v.pb.b, o); v.pb.x = ds(v.pb.x, o);
    v.pb.r = vs(v.pb.r, o); v.pb.e = vs(v.pb.e, o); v.pb.z = vs(v.pb.z, o); v.pb.q = vs(v.pb.q, o);
    v.pb.pv = vs(v.pb.pv, o); v.pb.pv1 = vs(v.pb.pv1, o);
    v.pb.refine_count = h->pb.refine_count ? h->pb.refine_count + m0 : nullptr;
    for (int l = 0; l < h->nlev; ++l) {
        const long long ol = (long long)m0 * h->lev[l].S;
        v.pb.lev_e[l] = vs(v.pb.lev_e[l], ol);
        v.pb.lev_f[l] = vs(v.pb.lev_f[l], ol);
        v.pb.lev_t[l] = vs(v.pb.lev_t[l], ol);
    }
    v.pt = h->pt;
    v.pt.part += (long long)m0 * h->pt.nblk;
    v.pt.red += m0;
    v.ctl = h->d_ctl + m0;
    v.ubc = h->d_ubc + (long long)m0 * h->g.ny;
    v.series = h->cfg.n_window > 0 ? h->d_series_slot + (long long)m0 * h->cfg.n_window * 8 : nullptr;
    v.u = ds(h->d_u, o); v.v = ds(h->d_v, o); v.us = ds(h->d_us, o); v.vs = ds(h->d_vs, o);
    v.p = ds(h->d_p, o); v.wf = ds(h->d_wf, 3 * o); v.wd = ds(h->d_wd, 3 * o);
    v.frect = ds(h->d_frect, (long long)m0 * 2 * h->nrect);
    v.Ru = vs(h->d_Ru, o); v.Rv = vs(h->d_Rv, o);
    return v;
}

// Member 0's arrays for the Welford of d = u - u_0 in the other members' correction.
static RefMember ref_member(envar_handle h)
{
    RefMember r{nullptr, nullptr, nullptr, nullptr};
    if (h->mixed || !h->d_wd) return r;
    if (h->batched) { r.us = h->d_us; r.vs = h->d_vs; r.x = h->pb.x; }
    else r.traj = h->d_traj;
    return r;
}

// One time step of M member slots starting at the view's first member, in three parts: the
// predictor and the pressure solve (part 0), the projection correction with the cost accumulation
// (part 1), and (FP64) the re-centring of the pressure increment, the next step's initial guess
// (part 2; the mixed path re-centres inside the correction and has no part 2).
static void enqueue_range(envar_handle h, int M, const MemberView &v, cudaStream_t st, int part)
{
    const Grid &g = h->g;
    const int want_wf = h->cfg.cost_mode == ENVAR_COST_DOMAIN ? 1 : 0;
    if (h->mixed) {
        if (part == 0) {
            launch_outflow_mx(g, M, v.ms, v.ubc, v.ctl, st);
            launch_predict_rhs_mx(g, h->mc, M, v.ms, v.ubc, h->d_inh, h->d_inl, v.ctl, v.pt.red, h->nfluid, st);
            launch_pressure_solve<float>(g, h->lev, M, v.pb, h->pc, v.pt, v.ctl, st);
        } else if (part == 1) {
            launch_correct_mx(g, h->mc, M, v.ms, h->ms, h->x0, h->y0, want_wf, v.series, v.pt, v.ctl, h->cfg.div_tol,
                              h->nfluid, st);
        }
        return;
    }
    if (part == 0) {
        launch_outflow(g, M, v.u, v.ubc, v.ctl, st);
        launch_predict<double>(g, M, v.u, v.v, v.p, (double *)v.Ru, (double *)v.Rv, v.us, v.vs, v.ubc, v.frect, v.ctl,
                               st);
        launch_rhs(g, M, v.us, v.vs, v.pb.b, v.ctl, st);
        launch_pressure_solve<double>(g, h->lev, M, v.pb, h->pc, v.pt, v.ctl, st);
    } else if (part == 1) {
        launch_correct(g, h->x0, h->y0, M, v.u, v.v, v.p, v.us, v.vs, v.pb.x, v.wf, v.wd, ref_member(h), want_wf,
                       v.series, v.pt, v.ctl, h->cfg.div_tol, h->nfluid, st);
    } else {
        launch_recenter(g, M, v.pb.x, v.pt, h->nfluid, st);
    }
}

// nsteps time steps of the first M member slots.  With all slots and several member groups, each
// group's steps form one chain on its side stream (a parallel branch of the captured graph, forked
// once and joined once), so one group's latency-bound phases overlap another's bandwidth-bound
// ones and the groups need not meet at every step.  The only coupling is member 0: the corrections
// of groups 1.. read its pressure increment and predictor (the exact DOMAIN contraction), so they
// wait for group 0's solve of the same step, and group 0 changes member 0's increment again (the
// FP64 re-centring, the mixed path's next initial guess) only after every group has read it.
static void enqueue_steps(envar_handle h, int M, int nsteps)
{
    const int G = (M == h->Mall) ? h->ngroups : 1;
    if (G <= 1) {
        const MemberView v = member_view(h, 0);
        for (int s = 0; s < nsteps; ++s)
            for (int part = 0; part < 3; ++part) enqueue_range(h, M, v, h->st, part);
        return;
    }
    const bool need_m0 = h->ms.wd != nullptr || h->d_wd != nullptr;
    const int per = (M + G - 1) / G;
    int ng = 0;
    while (ng < G && ng * per < M) ++ng;
    cudaEventRecord(h->ev_fork, h->st);
    for (int k = 0; k < ng; ++k) cudaStreamWaitEvent(h->side[k], h->ev_fork, 0);
    for (int s = 0; s < nsteps; ++s) {
        for (int k = 0; k < ng; ++k) {
            const int m0 = k * per, Mg = std::min(per, M - m0);
            const MemberView v = member_view(h, m0);
            if (need_m0 && k == 0 && s > 0)   // the previous step's corrections have read member 0
                for (int q = 1; q < ng; ++q) cudaStreamWaitEvent(h->side[0], h->ev_corr[q], 0);
            enqueue_range(h, Mg, v, h->side[k], 0);
            if (need_m0) {
                if (k == 0) cudaEventRecord(h->ev_solved0, h->side[0]);
                else cudaStreamWaitEvent(h->side[k], h->ev_solved0, 0);
            }
            enqueue_range(h, Mg, v, h->side[k], 1);
            if (need_m0 && k > 0) cudaEventRecord(h->ev_corr[k], h->side[k]);
        }
        for (int k = 0; k < ng; ++k) {
            const int m0 = k * per, Mg = std::min(per, M - m0);
            if (k == 0 && need_m0)
                for (int q = 1; q < ng; ++q) cudaStreamWaitEvent(h->side[0], h->ev_corr[q], 0);
            enqueue_range(h, Mg, member_view(h, m0), h->side[k], 2);
        }
    }
    for (int k = 0; k < ng; ++k) {
        cudaEventRecord(h->ev_join[k], h->side[k]);
        cudaStreamWaitEvent(h->st, h->ev_join[k], 0);
    }
}

static int capture(envar_handle h, int M, int nsteps, cudaGraphExec_t *out, long long *kernels)
{
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
    set_capturing(true);
    enqueue_steps(h, M, nsteps);
    set_capturing(false);
    cudaError_t e = cudaStreamEndCapture(h->st, &graph);
    if (e != cudaSuccess || capture_failed()) {
        if (e == cudaSuccess) cudaGraphDestroy(graph);
        set_err(h, "graph capture failed: %s", e != cudaSuccess ? cudaGetErrorString(e) : "conditional loop body");
        return ENVAR_ECUDA;
    }
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
    long long nk = 0;
    for (size_t k = 0; k < nn; ++k) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[k], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
    }
    *kernels = nk;
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        set_err(h, "graph instantiate failed: %s", cudaGetErrorString(e));
        return ENVAR_ECUDA;
    }
    return ENVAR_OK;
}

static int run_steps(envar_handle h, int M, int nsteps)
{
    GraphSet &gs = h->graphs[M == h->Mall ? 0 : 1];
    const int K = h->cfg.steps_per_graph;
    if (!gs.many) { int rc = capture(h, M, K, &gs.many, &gs.kernels_many); if (rc) return rc; }
    if (!gs.one) { int rc = capture(h, M, 1, &gs.one, &gs.kernels_one); if (rc) return rc; }
    int done = 0;
    for (; done + K <= nsteps; done += K) {
        CK(cudaGraphLaunch(gs.many, h->st));
        g_graph_kernels += gs.kernels_many;
    }
    for (; done < nsteps; ++done) {
        CK(cudaGraphLaunch(gs.one, h->st));
        g_graph_kernels += gs.kernels_one;
    }
    return ENVAR_OK;
}

// Load the initial state into the first M slots; slot k then holds ensemble member base + k.
static void reset_members(envar_handle h, int M, int base = 0)
{
    if (h->mixed) {
        launch_reset_mx(h->g, M, h->ic, h->ms, h->d_ctl, h->cfg.cost_mode == ENVAR_COST_DOMAIN ? 1 : 0, h->st);
    } else {
        launch_reset(h->g, M, h->d_u0, h->d_v0, h->d_u, h->d_v, h->d_p, h->pb.x, h->d_Ru, h->d_Rv,
                     h->tend_bytes / h->Mall * M, h->d_wf, h->d_wd, h->cfg.cost_mode == ENVAR_COST_DOMAIN ? 1 : 0,
                     h->d_ctl, h->st);
    }
    launch_set_gidx(h->d_ctl, M, base, h->st);
}

static void enqueue_cost(envar_handle h, int M, double *Jd, double *Js, double *Yd)
{
    const double *ser = h->cfg.n_window > 0 ? h->d_series_slot : nullptr;
    if (h->mixed) {
        const int nparts = 64;
        const long long S = h->g.S;
        double *part_d = h->d_costpart + (long long)nparts * M;
        if (h->ms.wf) launch_plane_partial_mx(h->g, M, h->ms.wf + 4 * S, h->ms.wf + 5 * S, 6 * S, h->d_costpart, nparts,
                                              h->st);
        if (h->ms.wd) launch_plane_partial_mx(h->g, M, h->ms.wd + 2 * S, h->ms.wd + 3 * S, 4 * S, part_d, nparts, h->st);
        launch_cost_final(h->g, M, h->ms.wf ? h->d_costpart : nullptr, h->ms.wd ? part_d : nullptr, nparts, ser, Jd,
                          Js, h->ms.wd ? Yd : nullptr, h->st);
    } else {
        launch_cost(h->g, M, h->d_wf, h->d_wd, ser, Jd, Js, Yd, h->d_costpart, h->st);
    }
}

// One forward evaluation of all N+1 members (batched) or of member `only` (plain, slot 0).
static int forward_members(envar_handle h)
{
    const int N = h->N;
    const int nw = std::max(h->cfg.n_window, 1);
    h->ctl_all.assign(N + 1, MemberCtl{});
    if (h->batched) {
        launch_member_forcing(h->Mall, 0, N, h->nrect, h->d_Erect, h->d_w, h->cfg.eps, h->d_frect, h->ms.frect,
                              h->st);
        reset_members(h, h->Mall);
        int rc = run_steps(h, h->Mall, h->cfg.n_steps);
        if (rc) return rc;
        enqueue_cost(h, h->Mall, h->d_Jd, h->d_Js, h->d_Yd);
        launch_copy_status(h->d_ctl, N + 1, h->d_status, h->st);
        CK(cudaMemcpyAsync(h->ctl_all.data(), h->d_ctl, sizeof(MemberCtl) * (N + 1), cudaMemcpyDeviceToHost, h->st));
    } else {
        for (int mm = 0; mm <= N; ++mm) {
            launch_member_forcing(1, mm, N, h->nrect, h->d_Erect, h->d_w, h->cfg.eps, h->d_frect, h->ms.frect,
                                  h->st);
            reset_members(h, 1, mm);
            int rc = run_steps(h, 1, h->cfg.n_steps);
            if (rc) return rc;
            enqueue_cost(h, 1, h->d_Jd + mm, h->d_Js + mm, h->d_Yd + mm);
            launch_copy_status(h->d_ctl, 1, h->d_status + mm, h->st);
            CK(cudaMemcpyAsync(h->d_series + (size_t)mm * nw * 8, h->d_series_slot, sizeof(double) * nw * 8,
                               cudaMemcpyDeviceToDevice, h->st));
            CK(cudaMemcpyAsync(&h->ctl_all[mm], h->d_ctl, sizeof(MemberCtl), cudaMemcpyDeviceToHost, h->st));
        }
        h->last_member_slot0 = N;
    }
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    h->have_forward = true;
    return ENVAR_OK;
}

// ------------------------------------------------------------------------------------ batches
// Several handles -- member groups of different grid sizes, Reynolds numbers and horizons -- advance
// together: one CUDA graph per chunk holds every handle's next c_k time steps as parallel branches
// (each handle's own member groups branch further inside), and c_k is proportional to the handle's
// horizon, so all handles finish on the same chunk.
struct envar_batch_s {
    std::vector<envar_handle> h;
    std::vector<int> per_chunk;       // time steps of each handle per chunk
    int n_chunks = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    cudaGraphExec_t graph = nullptr;
    long long graph_kernels = 0;
    cudaEvent_t ev = nullptr;
    std::vector<cudaEvent_t> ev_h;
};

static long long gcd_ll(long long a, long long b) { while (b) { long long t = a % b; a = b; b = t; } return a; }

// ------------------------------------------------------------------------------------ API
extern "C" int envar_init(envar_handle *out, const envar_config *cfg, void *cuda_stream)
{
    if (!out || !cfg) {
        set_err(nullptr, "envar_init: null argument");
        return ENVAR_EINVAL;
    }
    *out = nullptr;
    const envar_config &c = *cfg;
    if (c.nx < 8 || c.ny < 4 || c.nx % 2 || c.ny % 2 || c.n_steps < 1 || c.n_window < 0 || c.n_window > c.n_steps ||
        c.n_members < 0 || !(c.Re > 0) || !(c.cfl > 0) || !(c.eps > 0) || !(c.sigma >= 0) || !(c.corr_len > 0) ||
        c.precision < 0 || c.precision > 2 || c.cost_mode < 0 || c.cost_mode > 1 || !(c.div_tol > 0) ||
        c.max_outer < 1 || c.max_inner < 1 || c.nu_pre < 1 || c.nu_pre > 3 || c.nu_post < 1 || c.nu_post > 3 ||
        c.coarse_sweeps < 1 || c.steps_per_graph < 1 || !(c.x1 > c.x0) || !(c.y1 > c.y0) || !(c.inner_rtol > 0) ||
        c.member_groups < 0 || c.member_groups > ENVAR_MAX_GROUPS || c.guess_extrapolation < 0 ||
        c.guess_extrapolation > 1 || c.nu_coarse < 0 || c.nu_coarse > 3) {
        set_err(nullptr, "envar_init: invalid configuration");
        return ENVAR_EINVAL;
    }
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        set_err(nullptr, "envar_init: no CUDA device");
        return ENVAR_EDEVICE;
    }
    if (!(prop.major == 10 && prop.minor == 3)) {
        set_err(nullptr, "envar_init: device %s is sm_%d%d; this library is built for sm_103a (GB300)", prop.name,
                prop.major, prop.minor);
        return ENVAR_EDEVICE;
    }
    envar_handle h = new envar_handle_s();
    h->cfg = c;
    h->N = c.n_members;
    h->batched = (c.precision != ENVAR_FP64_PLAIN);
    h->mixed = (c.precision == ENVAR_MIXED);
    h->Mall = h->batched ? h->N + 1 : 1;
    if (cuda_stream) {
        h->st = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking) != cudaSuccess) {
            set_err(nullptr, "envar_init: stream creation failed");
            delete h;
            return ENVAR_ECUDA;
        }
        h->own_stream = true;
    }
    {   // member groups: side streams and fork / join events for the captured step
        int G = c.member_groups ? c.member_groups : (h->Mall >= 24 ? 4 : (h->Mall >= 8 ? 2 : 1));
        if (!h->batched) G = 1;
        h->ngroups = std::max(1, std::min(G, h->Mall));
        if (h->ngroups > 1) {
            bool ok = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
                      cudaEventCreateWithFlags(&h->ev_solved0, cudaEventDisableTiming) == cudaSuccess;
            for (int k = 0; ok && k < h->ngroups; ++k)
                ok = cudaStreamCreateWithFlags(&h->side[k], cudaStreamNonBlocking) == cudaSuccess &&
                     cudaEventCreateWithFlags(&h->ev_join[k], cudaEventDisableTiming) == cudaSuccess &&
                     cudaEventCreateWithFlags(&h->ev_corr[k], cudaEventDisableTiming) == cudaSuccess;
            if (!ok) {
                set_err(nullptr, "envar_init: stream or event creation failed");
                envar_destroy(h);
                return ENVAR_ECUDA;
            }
        }
    }
    int rc = build_geometry(h);
    if (!rc) rc = alloc_buffers(h);
    if (!rc) {
        PoissonCfg &pc = h->pc;
        pc.nlev = h->nlev; pc.ncoarse = h->ncoarse;
        pc.nu_pre = c.nu_pre; pc.nu_post = c.nu_post; pc.coarse_sweeps = c.coarse_sweeps;
        pc.nu_c = c.nu_coarse;
        pc.max_outer = c.max_outer; pc.max_inner = c.max_inner;
        pc.inner_rtol2 = c.inner_rtol * c.inner_rtol;
        pc.rtol_abs = c.div_tol * h->g.hxy / h->g.dt;
        pc.cimg = h->d_cimg;
        pc.cimg_bytes = h->cimg_bytes;
        {
            const Grid &g = h->g;
            auto split = [](double d, float *hi, float *lo) { *hi = (float)d; *lo = (float)(d - (double)*hi); };
            MixConst &K = h->mc;
            double gx = g.dt / g.dx, gy = g.dt / g.dy, kx = g.dy / g.dt, ky = g.dx / g.dt;
            split(gx, &K.gxh, &K.gxl); split(gy, &K.gyh, &K.gyl);
            split(kx, &K.kxh, &K.kxl); split(ky, &K.kyh, &K.kyl);
            split(kx * gx, &K.cxh, &K.cxl); split(ky * gy, &K.cyh, &K.cyl);
            K.dt = (float)g.dt; K.gxf = (float)gx; K.gyf = (float)gy;
            K.i4dx = (float)(0.25 / g.dx); K.i4dy = (float)(0.25 / g.dy);
            K.nudx2 = (float)(g.nu / (g.dx * g.dx)); K.nudy2 = (float)(g.nu / (g.dy * g.dy));
            K.dxf = (float)g.dx; K.dyf = (float)g.dy;
            pc.df_outer = h->mixed ? 1 : 0;
            pc.conditional_loop = c.conditional_refinement ? 1 : 0;
            pc.mc = K;
        }
        if (h->mixed) prepare_poisson_kernels<float>(); else prepare_poisson_kernels<double>();
        rc = generate_ensemble(h);
    }
    if (rc) {
        std::snprintf(g_init_err, sizeof(g_init_err), "%s", h->err);
        envar_destroy(h);
        return rc;
    }
    *out = h;
    return ENVAR_OK;
}

extern "C" int envar_destroy(envar_handle h)
{
    if (!h) return ENVAR_OK;
    if (h->st) cudaStreamSynchronize(h->st);
    for (auto &gs : h->graphs) {
        if (gs.many) cudaGraphExecDestroy(gs.many);
        if (gs.one) cudaGraphExecDestroy(gs.one);
    }
    for (auto &row : h->adj_graph)
        for (auto &ge : row)
            if (ge) cudaGraphExecDestroy(ge);
    for (void *p : h->allocs) cudaFree(p);
    if (h->d_snap) cudaFree(h->d_snap);
    for (int k = 0; k < ENVAR_MAX_GROUPS; ++k) {
        if (h->side[k]) cudaStreamDestroy(h->side[k]);
        if (h->ev_join[k]) cudaEventDestroy(h->ev_join[k]);
        if (h->ev_corr[k]) cudaEventDestroy(h->ev_corr[k]);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_solved0) cudaEventDestroy(h->ev_solved0);
    if (h->own_stream) cudaStreamDestroy(h->st);
    delete h;
    return ENVAR_OK;
}

extern "C" const char *envar_last_error(envar_handle h) { return h ? h->err : g_init_err; }

extern "C" int envar_sizes(envar_handle h, int *n_ctrl, int *n_cc, int *n_levels, double *dt)
{
    if (!h) return ENVAR_EINVAL;
    if (n_ctrl) *n_ctrl = h->n_ctrl;
    if (n_cc) *n_cc = h->ncc;
    if (n_levels) *n_levels = h->nlev;
    if (dt) *dt = h->g.dt;
    return ENVAR_OK;
}

extern "C" int envar_set_initial_state(envar_handle h, const double *u0, const double *v0)
{
    if (!h || !u0 || !v0) return ENVAR_EINVAL;
    if (h->mixed) {
        launch_load_ic_mx(h->g, u0, v0, h->ic, h->st);
    } else {
        CK(cudaMemsetAsync(h->d_u0, 0, sizeof(double) * h->g.S, h->st));
        CK(cudaMemsetAsync(h->d_v0, 0, sizeof(double) * h->g.S, h->st));
        launch_load_ic(h->g, u0, v0, h->d_u0, h->d_v0, h->st);
    }
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    h->have_ic = true;
    return ENVAR_OK;
}

extern "C" int envar_set_ensemble(envar_handle h, const double *E, int n_ctrl, int N)
{
    if (!h || !E) return ENVAR_EINVAL;
    if (n_ctrl != h->n_ctrl || N != h->N) {
        set_err(h, "envar_set_ensemble: expected %d x %d, got %d x %d", h->n_ctrl, h->N, n_ctrl, N);
        return ENVAR_EINVAL;
    }
    CK(cudaMemcpyAsync(h->d_E, E, sizeof(double) * (size_t)n_ctrl * N, cudaMemcpyDeviceToDevice, h->st));
    launch_compact_to_rect(N, h->nrect, h->ncc, h->d_cidx, h->d_E, h->d_Erect, h->st);
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    return ENVAR_OK;
}

extern "C" int envar_get_ensemble(envar_handle h, double *E)
{
    if (!h || !E) return ENVAR_EINVAL;
    CK(cudaMemcpyAsync(E, h->d_E, sizeof(double) * (size_t)h->n_ctrl * h->N, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
    return ENVAR_OK;
}

extern "C" int envar_batch_create(envar_batch *out, envar_handle *handles, int n, void *cuda_stream)
{
    if (!out || !handles || n < 1) return ENVAR_EINVAL;
    *out = nullptr;
    long long g = 0;
    int min_steps = 0;
    for (int k = 0; k < n; ++k) {
        envar_handle h = handles[k];
        if (!h || !h->batched) {
            set_err(nullptr, "envar_batch_create: handle %d is missing or not batched (FP64_PLAIN)", k);
            return ENVAR_EINVAL;
        }
        for (int j = 0; j < k; ++j)
            if (handles[j] == h) { set_err(nullptr, "envar_batch_create: handle %d appears twice", k); return ENVAR_EINVAL; }
        g = gcd_ll(g, h->cfg.n_steps);
        min_steps = k ? std::min(min_steps, h->cfg.n_steps) : h->cfg.n_steps;
    }
    // the fewest chunks (largest graphs) that keep at least 10 steps of the shortest horizon per chunk
    long long chunks = g;
    for (long long d = 1; d <= g; ++d)
        if (g % d == 0 && min_steps / (g / d) >= std::min(10, min_steps)) { chunks = g / d; break; }
    int maxc = 0;
    for (int k = 0; k < n; ++k) maxc = std::max<long long>(maxc, handles[k]->cfg.n_steps / chunks);
    if (maxc > 400) {
        set_err(nullptr, "envar_batch_create: horizons share too small a common step (%lld chunks, %d steps per chunk)",
                chunks, maxc);
        return ENVAR_EINVAL;
    }
    envar_batch b = new envar_batch_s();
    b->h.assign(handles, handles + n);
    b->n_chunks = (int)chunks;
    for (int k = 0; k < n; ++k) b->per_chunk.push_back((int)(handles[k]->cfg.n_steps / chunks));
    if (cuda_stream) b->st = (cudaStream_t)cuda_stream;
    else if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) == cudaSuccess) b->own_stream = true;
    bool ok = b->st && cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) == cudaSuccess;
    b->ev_h.assign(n, nullptr);
    for (int k = 0; ok && k < n; ++k) ok = cudaEventCreateWithFlags(&b->ev_h[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        set_err(nullptr, "envar_batch_create: stream or event creation failed");
        envar_batch_destroy(b);
        return ENVAR_ECUDA;
    }
    *out = b;
    return ENVAR_OK;
}

extern "C" int envar_batch_destroy(envar_batch b)
{
    if (!b) return ENVAR_OK;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->ev) cudaEventDestroy(b->ev);
    for (cudaEvent_t e : b->ev_h) if (e) cudaEventDestroy(e);
    if (b->own_stream) cudaStreamDestroy(b->st);
    delete b;
    return ENVAR_OK;
}

// One chunk: every handle's next per_chunk[k] steps, forked from and joined to the batch stream.
static int batch_capture(envar_batch b)
{
    envar_handle h0 = b->h[0];
    cudaGraph_t graph;
    cudaError_t e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { set_err(h0, "batch capture: %s", cudaGetErrorString(e)); return ENVAR_ECUDA; }
    set_capturing(true);
    cudaEventRecord(b->ev, b->st);
    for (size_t k = 0; k < b->h.size(); ++k) {
        envar_handle h = b->h[k];
        cudaStreamWaitEvent(h->st, b->ev, 0);
        enqueue_steps(h, h->Mall, b->per_chunk[k]);
        cudaEventRecord(b->ev_h[k], h->st);
        cudaStreamWaitEvent(b->st, b->ev_h[k], 0);
    }
    set_capturing(false);
    e = cudaStreamEndCapture(b->st, &graph);
    if (e != cudaSuccess || capture_failed()) {
        if (e == cudaSuccess) cudaGraphDestroy(graph);
        set_err(h0, "batch capture failed: %s", e != cudaSuccess ? cudaGetErrorString(e) : "conditional loop body");
        return ENVAR_ECUDA;
    }
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
    b->graph_kernels = 0;
    for (size_t k = 0; k < nn; ++k) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[k], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++b->graph_kernels;
    }
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { b->graph = nullptr; set_err(h0, "batch graph instantiate: %s", cudaGetErrorString(e)); return ENVAR_ECUDA; }
    return ENVAR_OK;
}

extern "C" int envar_batch_forward(envar_batch b, const double *const *w_devs)
{
    if (!b || !w_devs) return ENVAR_EINVAL;
    for (envar_handle h : b->h)
        if (!h->have_ic) { set_err(h, "envar_batch_forward: no initial state"); return ENVAR_ESTATE; }
    // the solver parameters of a handle may have changed (envar_autotune): recapture then
    if (!b->graph) { int rc = batch_capture(b); if (rc) return rc; }
    for (size_t k = 0; k < b->h.size(); ++k) {
        envar_handle h = b->h[k];
        h->ctl_all.assign(h->N + 1, MemberCtl{});
        if (h->N > 0) {
            if (!w_devs[k]) return ENVAR_EINVAL;
            CK(cudaMemcpyAsync(h->d_w, w_devs[k], sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->st));
        }
        launch_member_forcing(h->Mall, 0, h->N, h->nrect, h->d_Erect, h->d_w, h->cfg.eps, h->d_frect, h->ms.frect,
                              h->st);
        reset_members(h, h->Mall);
        CK(cudaEventRecord(b->ev_h[k], h->st));
        CK(cudaStreamWaitEvent(b->st, b->ev_h[k], 0));
    }
    envar_handle h = b->h[0];   // error messages of the batch's own stream work go to the first handle
    for (int c = 0; c < b->n_chunks; ++c) {
        CK(cudaGraphLaunch(b->graph, b->st));
        g_graph_kernels += b->graph_kernels;
    }
    CK(cudaEventRecord(b->ev, b->st));
    for (envar_handle hk : b->h) {
        h = hk;
        CK(cudaStreamWaitEvent(h->st, b->ev, 0));
        enqueue_cost(h, h->Mall, h->d_Jd, h->d_Js, h->d_Yd);
        launch_copy_status(h->d_ctl, h->N + 1, h->d_status, h->st);
        CK(cudaMemcpyAsync(h->ctl_all.data(), h->d_ctl, sizeof(MemberCtl) * (h->N + 1), cudaMemcpyDeviceToHost, h->st));
    }
    for (envar_handle hk : b->h) {
        h = hk;
        CK(cudaStreamSynchronize(h->st));
        h->have_forward = true;
    }
    CK(cudaGetLastError());
    return ENVAR_OK;
}

extern "C" int envar_batch_info(envar_batch b, int *n_chunks, int *steps_per_chunk)
{
    if (!b) return ENVAR_EINVAL;
    if (n_chunks) *n_chunks = b->n_chunks;
    if (steps_per_chunk)
        for (size_t k = 0; k < b->per_chunk.size(); ++k) steps_per_chunk[k] = b->per_chunk[k];
    return ENVAR_OK;
}

extern "C" int envar_eigen_ensemble(envar_handle h, double *lambda_host)
{
    if (!h) return ENVAR_EINVAL;
    const int N = h->N;
    if (N < 1) { set_err(h, "envar_eigen_ensemble: ensemble is empty"); return ENVAR_EINVAL; }
    const int y_only = h->cfg.forcing_y_only ? 1 : 0;
    const int k = y_only ? N : (N + 1) / 2;
    if (k > h->ncc) { set_err(h, "envar_eigen_ensemble: %d eigenvectors requested, %d control cells", k, h->ncc); return ENVAR_EINVAL; }
    // Lanczos steps: from max(2k + 40, 64), doubling while a kept Ritz pair is not converged, up to
    // the control cells or 768 (the projected matrix is diagonalised in one block)
    int mmax = std::min(h->ncc, 768);
    mmax -= mmax % 2;
    const int m0 = std::min(mmax, std::max(2 * k + 40, 64));
    if (mmax < k + 2) { set_err(h, "envar_eigen_ensemble: too few control cells for %d eigenvectors", k); return ENVAR_EINVAL; }
    const size_t nd = eigen_work_doubles(h->nrx, h->nry, h->ncc, mmax, k);
    void *work = nullptr;
    cudaError_t e = cudaMalloc(&work, sizeof(double) * nd);
    if (e != cudaSuccess) { set_err(h, "envar_eigen_ensemble: %zu bytes of work space: %s", sizeof(double) * nd, cudaGetErrorString(e)); return ENVAR_ENOMEM; }
    std::vector<double> lam((size_t)k);
    int steps = 0;
    double bound = 0.0;
    const double tol = 1e-12;
    int rc = eigen_ensemble(h->nrx, h->nry, h->g.dx, h->g.dy, h->cfg.corr_len, h->cfg.sigma, h->ncc, h->d_cidx, N,
                            y_only, m0, mmax, tol, h->cfg.seed, (double *)work, h->d_E, lam.data(), &steps, &bound,
                            h->st);
    if (!rc) launch_compact_to_rect(N, h->nrect, h->ncc, h->d_cidx, h->d_E, h->d_Erect, h->st);
    e = cudaStreamSynchronize(h->st);
    cudaFree(work);
    if (rc) { set_err(h, "envar_eigen_ensemble: bad Lanczos size"); return ENVAR_EINVAL; }
    if (e != cudaSuccess) { set_err(h, "envar_eigen_ensemble: %s", cudaGetErrorString(e)); return ENVAR_ECUDA; }
    CK(cudaGetLastError());
    if (bound > tol) {
        set_err(h, "envar_eigen_ensemble: Ritz residual %g after %d Lanczos steps (relative to the largest eigenvalue)",
                bound, steps);
        return ENVAR_ESTATE;
    }
    if (lambda_host)
        for (int i = 0; i < N; ++i) lambda_host[i] = lam[(size_t)(y_only ? i : i / 2)];
    h->have_forward = false;
    return ENVAR_OK;
}

extern "C" int envar_forward_ensemble(envar_handle h, const double *w)
{
    if (!h) return ENVAR_EINVAL;
    if (!h->have_ic) { set_err(h, "envar_forward_ensemble: no initial state"); return ENVAR_ESTATE; }
    if (h->N > 0) {
        if (!w) return ENVAR_EINVAL;
        CK(cudaMemcpyAsync(h->d_w, w, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->st));
    }
    return forward_members(h);
}

extern "C" int envar_cost(envar_handle h, double *J, double *Jprior)
{
    if (!h) return ENVAR_EINVAL;
    if (!h->have_forward) { set_err(h, "envar_cost: no forward run"); return ENVAR_ESTATE; }
    const double *src = (h->cfg.cost_mode == ENVAR_COST_SENSORS) ? h->d_Js : h->d_Jd;
    if (J) CK(cudaMemcpyAsync(J, src, sizeof(double) * (h->N + 1), cudaMemcpyDeviceToHost, h->st));
    if (Jprior) {
        if (h->N > 0) {
            launch_scalar_gradient(h->N, src, h->d_w, h->cfg.eps, h->d_status, h->d_gscalar, h->d_jprior, h->st);
            CK(cudaMemcpyAsync(Jprior, h->d_jprior, sizeof(double), cudaMemcpyDeviceToHost, h->st));
        } else {
            *Jprior = 0.0;
        }
    }
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    return ENVAR_OK;
}

// Eq. (gradient_EnVar) for the last forward run, on the device: the scalar-anomaly form and the
// prior cost always (d_gscalar, d_jprior), and the explicit contraction Y^T (Hq_0 - y) + (N-1) w of
// the configured observation operator in d_g.  Members whose status word is nonzero contribute
// no column of Y.
static void compute_gradient(envar_handle h)
{
    const bool sensors = h->cfg.cost_mode == ENVAR_COST_SENSORS;
    const double *src = sensors ? h->d_Js : h->d_Jd;
    launch_scalar_gradient(h->N, src, h->d_w, h->cfg.eps, h->d_status, h->d_gscalar, h->d_jprior, h->st);
    if (sensors && h->cfg.n_window > 0)
        launch_sensor_gradient(h->N, h->cfg.n_window, h->d_series, h->cfg.eps, h->d_w, h->d_status, h->d_g, h->st);
    else if (!sensors && h->cfg.n_window > 0)
        launch_domain_gradient(h->N, h->d_Jd, h->d_Yd, h->d_w, h->cfg.eps, h->d_status, h->d_g, h->st);
    else
        cudaMemcpyAsync(h->d_g, h->d_gscalar, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->st);
}

static int check_member0(envar_handle h, const char *what)
{
    if (!h->ctl_all.empty() && h->ctl_all[0].status != 0) {
        set_err(h, "%s: the unperturbed member failed (status 0x%x); no gradient", what, h->ctl_all[0].status);
        return ENVAR_ESTATE;
    }
    return ENVAR_OK;
}

extern "C" int envar_gradient(envar_handle h, double *g, double *df)
{
    if (!h) return ENVAR_EINVAL;
    if (!h->have_forward) { set_err(h, "envar_gradient: no forward run"); return ENVAR_ESTATE; }
    if (h->N < 1) { set_err(h, "envar_gradient: ensemble is empty"); return ENVAR_ESTATE; }
    if (int rc = check_member0(h, "envar_gradient")) return rc;
    compute_gradient(h);
    if (df) launch_df(h->N, h->n_ctrl, h->d_E, h->d_g, 1.0 / std::max(h->N - 1, 1), df, h->st);
    if (g) CK(cudaMemcpyAsync(g, h->d_g, sizeof(double) * h->N, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    return ENVAR_OK;
}

extern "C" int envar_gradient_scalar(envar_handle h, double *g)
{
    if (!h || !g) return ENVAR_EINVAL;
    if (!h->have_forward) { set_err(h, "envar_gradient_scalar: no forward run"); return ENVAR_ESTATE; }
    if (h->N < 1) { set_err(h, "envar_gradient_scalar: ensemble is empty"); return ENVAR_ESTATE; }
    if (int rc = check_member0(h, "envar_gradient_scalar")) return rc;
    compute_gradient(h);
    CK(cudaMemcpyAsync(g, h->d_gscalar, sizeof(double) * h->N, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    return ENVAR_OK;
}

extern "C" int envar_excluded_members(envar_handle h, int *count)
{
    if (!h || !count) return ENVAR_EINVAL;
    if (!h->have_forward) { set_err(h, "envar_excluded_members: no forward run"); return ENVAR_ESTATE; }
    int n = 0;
    for (int m = 1; m <= h->N; ++m) n += h->ctl_all[m].status != 0;
    *count = n;
    return ENVAR_OK;
}

extern "C" int envar_step(envar_handle h, double alpha, double *w_inout, double *J0_out)
{
    if (!h || !w_inout) return ENVAR_EINVAL;
    if (!h->have_ic) { set_err(h, "envar_step: no initial state"); return ENVAR_ESTATE; }
    if (h->N < 1) { set_err(h, "envar_step: ensemble is empty"); return ENVAR_ESTATE; }
    CK(cudaMemcpyAsync(h->d_w, w_inout, sizeof(double) * h->N, cudaMemcpyHostToDevice, h->st));
    int rc = forward_members(h);
    if (rc) return rc;
    if ((rc = check_member0(h, "envar_step"))) return rc;
    compute_gradient(h);
    double J0 = 0.0, jp = 0.0;
    const double *src = (h->cfg.cost_mode == ENVAR_COST_SENSORS) ? h->d_Js : h->d_Jd;
    CK(cudaMemcpyAsync(&J0, src, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(&jp, h->d_jprior, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    launch_update_w(h->N, h->d_w, h->d_g, alpha / std::max(h->N - 1, 1), h->st);
    CK(cudaMemcpyAsync(w_inout, h->d_w, sizeof(double) * h->N, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    if (J0_out) *J0_out = J0 + jp;
    return ENVAR_OK;
}

extern "C" int envar_step_device(envar_handle h, double alpha, double *w_inout, double *J0_out)
{
    if (!h || !w_inout) return ENVAR_EINVAL;
    if (!h->have_ic) { set_err(h, "envar_step_device: no initial state"); return ENVAR_ESTATE; }
    if (h->N < 1) { set_err(h, "envar_step_device: ensemble is empty"); return ENVAR_ESTATE; }
    CK(cudaMemcpyAsync(h->d_w, w_inout, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->st));
    int rc = forward_members(h);
    if (rc) return rc;
    compute_gradient(h);
    if (J0_out) {
        const double *src = (h->cfg.cost_mode == ENVAR_COST_SENSORS) ? h->d_Js : h->d_Jd;
        launch_total_cost(src, h->d_jprior, J0_out, h->st);
    }
    launch_update_w(h->N, h->d_w, h->d_g, alpha / std::max(h->N - 1, 1), h->st);
    CK(cudaMemcpyAsync(w_inout, h->d_w, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaGetLastError());
    return ENVAR_OK;
}

// ------------------------------------------------------------------------------------ optimisers
// Sec. 3.3.1: Gauss-Newton with H_GN = Y^T Y + (N-1) I (Eq. Hessian_EnVar, update_Newton) on the
// sensor-space Y of Eq. (fdapprox), and L-BFGS (Eq. update_BFGS) with an Armijo line search.

static int gn_buffers(envar_handle h)
{
    if (h->d_Y) return ENVAR_OK;
    const int N = h->N;
    const long long nobs = 8LL * h->cfg.n_window;
    DA(h->d_Y, (size_t)N * nobs); DA(h->d_h0, nobs); DA(h->d_smean, (size_t)(N + 1) * 8);
    DA(h->d_H, (size_t)N * N); DA(h->d_L, (size_t)N * N); DA(h->d_x, N); DA(h->d_info, 1);
    return ENVAR_OK;
}

// H_GN and g of the last forward run into d_H, d_g (device).
static int gn_assemble(envar_handle h)
{
    if (int rc = gn_buffers(h)) return rc;
    const long long nobs = 8LL * h->cfg.n_window;
    launch_sensor_anomalies(h->N, h->cfg.n_window, h->d_series, h->cfg.eps, h->d_status, h->d_smean, h->d_Y, h->d_h0,
                            h->st);
    launch_gram(h->N, nobs, h->d_Y, h->d_h0, h->d_w, h->d_H, h->d_g, h->st);
    return ENVAR_OK;
}

static int gn_check(envar_handle h, const char *what)
{
    if (h->cfg.cost_mode != ENVAR_COST_SENSORS || h->cfg.n_window < 1 || h->N < 1) {
        set_err(h, "%s: Gauss-Newton needs the SENSORS observation operator, n_window >= 1 and N >= 1", what);
        return ENVAR_EINVAL;
    }
    return ENVAR_OK;
}

extern "C" int envar_gn_hessian(envar_handle h, double *H_host)
{
    if (!h || !H_host) return ENVAR_EINVAL;
    if (int rc = gn_check(h, "envar_gn_hessian")) return rc;
    if (!h->have_forward) { set_err(h, "envar_gn_hessian: no forward run"); return ENVAR_ESTATE; }
    if (int rc = gn_assemble(h)) return rc;
    CK(cudaMemcpyAsync(H_host, h->d_H, sizeof(double) * h->N * h->N, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    return ENVAR_OK;
}

extern "C" int envar_gn_step(envar_handle h, double alpha, double *w_inout, double *J0_out)
{
    if (!h || !w_inout) return ENVAR_EINVAL;
    if (int rc = gn_check(h, "envar_gn_step")) return rc;
    if (!h->have_ic) { set_err(h, "envar_gn_step: no initial state"); return ENVAR_ESTATE; }
    CK(cudaMemcpyAsync(h->d_w, w_inout, sizeof(double) * h->N, cudaMemcpyHostToDevice, h->st));
    int rc = forward_members(h);
    if (rc) return rc;
    if ((rc = check_member0(h, "envar_gn_step"))) return rc;
    compute_gradient(h);   // J_prior; d_g is rebuilt by the Gram kernel (same contraction)
    if ((rc = gn_assemble(h))) return rc;
    launch_cholesky_step(h->N, h->d_H, h->d_L, h->d_g, h->d_w, alpha, h->d_x, h->d_wt, h->d_info, h->st);
    double J0 = 0.0, jp = 0.0;
    int info = 0;
    CK(cudaMemcpyAsync(&J0, h->d_Js, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(&jp, h->d_jprior, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(&info, h->d_info, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (info != 0) {
        set_err(h, "envar_gn_step: H_GN is not positive definite (pivot %d)", info);
        return ENVAR_ESTATE;
    }
    CK(cudaMemcpyAsync(h->d_w, h->d_wt, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(w_inout, h->d_w, sizeof(double) * h->N, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    if (J0_out) *J0_out = J0 + jp;
    return ENVAR_OK;
}

static int lb_setup(envar_handle h, LbfgsState &L, int n, int m)
{
    if (L.m != m || L.n != n) {
        DA(L.S, (size_t)m * n); DA(L.Y, (size_t)m * n); DA(L.sy, 2 * m); DA(L.a, m); DA(L.order, m);
        DA(L.q, n); DA(L.p, n); DA(L.gp, 1); DA(L.xprev, n); DA(L.gprev, n);
        L.m = m;
        L.n = n;
    }
    L.count = 0;
    L.head = 0;
    L.have_prev = false;
    return ENVAR_OK;
}

// The pair (x - x_prev, g - g_prev) joins the history when its curvature s^T y is positive.
static int lb_update(envar_handle h, LbfgsState &L, const double *x, const double *g)
{
    if (!L.have_prev) return ENVAR_OK;
    const int slot = L.head;
    launch_lbfgs_pair(L.n, x, L.xprev, g, L.gprev, slot, L.S, L.Y, L.sy, L.m, h->st);
    double sy[2] = {0.0, 0.0};
    CK(cudaMemcpyAsync(&sy[0], L.sy + slot, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(&sy[1], L.sy + L.m + slot, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (sy[0] > 1e-10 * std::sqrt(sy[1])) {
        L.head = (L.head + 1) % L.m;
        L.count = std::min(L.count + 1, L.m);
    }
    return ENVAR_OK;
}

// p = -H g by the two-loop recursion (initial matrix (s^T y / y^T y) I, or gamma0 I without pairs);
// *gp_host = g^T p.  Then x_prev, g_prev <- x, g.
static int lb_direction(envar_handle h, LbfgsState &L, const double *x, const double *g, double gamma0, double *gp_host)
{
    std::vector<int> order((size_t)L.count);
    for (int r = 0; r < L.count; ++r) order[r] = (L.head - L.count + r + L.m) % L.m;
    if (L.count) CK(cudaMemcpyAsync(L.order, order.data(), sizeof(int) * L.count, cudaMemcpyHostToDevice, h->st));
    launch_lbfgs_direction(L.n, L.count, L.order, L.S, L.Y, g, gamma0, L.q, L.a, L.p, L.gp, h->st);
    CK(cudaMemcpyAsync(L.xprev, x, sizeof(double) * L.n, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(L.gprev, g, sizeof(double) * L.n, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(gp_host, L.gp, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return ENVAR_OK;
}

extern "C" int envar_lbfgs_reset(envar_handle h, int memory)
{
    if (!h || memory < 1 || memory > 64 || h->N < 1) return ENVAR_EINVAL;
    if (!h->d_prior_t) DA(h->d_prior_t, 1);
    return lb_setup(h, h->lbw, h->N, memory);
}

// J(w_t) = J_obs of member 0 alone with forcing E w_t, plus the prior (N-1)/2 w_t^T w_t (Eq. J_w).
static int trial_cost(envar_handle h, const double *wt, double *J)
{
    launch_member_forcing(1, 0, h->N, h->nrect, h->d_Erect, wt, h->cfg.eps, h->d_frect, h->ms.frect, h->st);
    reset_members(h, 1);
    int rc = run_steps(h, 1, h->cfg.n_steps);
    if (rc) return rc;
    enqueue_cost(h, 1, h->d_Jd_slot, h->d_Js_slot, h->d_Yd_slot);
    const double *src = (h->cfg.cost_mode == ENVAR_COST_SENSORS) ? h->d_Js_slot : h->d_Jd_slot;
    double jo = 0.0, jp = 0.0;
    MemberCtl c0{};
    CK(cudaMemcpyAsync(&jo, src, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(&jp, h->d_prior_t, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(&c0, h->d_ctl, sizeof(MemberCtl), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    *J = (c0.status != 0) ? HUGE_VAL : jo + jp;   // a failed trial run is rejected by the line search
    return ENVAR_OK;
}

extern "C" int envar_lbfgs_step(envar_handle h, double *w_inout, double *J0_out, double *alpha_out, int *evals_out)
{
    if (!h || !w_inout) return ENVAR_EINVAL;
    if (!h->have_ic) { set_err(h, "envar_lbfgs_step: no initial state"); return ENVAR_ESTATE; }
    if (h->N < 1) { set_err(h, "envar_lbfgs_step: ensemble is empty"); return ENVAR_ESTATE; }
    int rc = 0;
    if (h->lbw.m == 0 && (rc = envar_lbfgs_reset(h, 8))) return rc;
    LbfgsState &L = h->lbw;
    const int N = h->N;
    CK(cudaMemcpyAsync(h->d_w, w_inout, sizeof(double) * N, cudaMemcpyHostToDevice, h->st));
    if ((rc = forward_members(h))) return rc;
    if ((rc = check_member0(h, "envar_lbfgs_step"))) return rc;
    compute_gradient(h);
    if ((rc = lb_update(h, L, h->d_w, h->d_g))) return rc;
    const double gamma0 = 1.0 / std::max(N - 1, 1);   // inverse of the prior Hessian (N-1) I
    double gp = 0.0;
    if ((rc = lb_direction(h, L, h->d_w, h->d_g, gamma0, &gp))) return rc;
    if (!(gp < 0.0)) {
        // not a descent direction: drop the history and take the prior-preconditioned gradient step
        L.count = 0;
        if ((rc = lb_direction(h, L, h->d_w, h->d_g, gamma0, &gp))) return rc;
    }
    const double *src = (h->cfg.cost_mode == ENVAR_COST_SENSORS) ? h->d_Js : h->d_Jd;
    double J0 = 0.0, jp = 0.0;
    CK(cudaMemcpyAsync(&J0, src, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(&jp, h->d_jprior, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    const double Jw = J0 + jp;
    // Armijo backtracking: J(w + a p) <= J(w) + c1 a g^T p, a = 1, 1/2, ...
    const double c1 = 1e-4;
    double a = 1.0, Jt = 0.0;
    int evals = 0;
    bool ok = false;
    for (int k = 0; k < 12; ++k) {
        launch_trial_point(N, h->d_w, L.p, a, h->d_wt, h->d_prior_t, h->st);
        if ((rc = trial_cost(h, h->d_wt, &Jt))) return rc;
        ++evals;
        ok = Jt <= Jw + c1 * a * gp;
        if (ok) break;
        a *= 0.5;
    }
    h->have_forward = false;   // slot 0 now holds the last trial run
    h->last_member_slot0 = -2;
    if (evals_out) *evals_out = evals;
    if (J0_out) *J0_out = Jw;
    if (!ok) {
        // no trial decreased J by the Armijo margin: w is stationary to the accuracy of J
        L.have_prev = false;
        if (alpha_out) *alpha_out = 0.0;
        return ENVAR_OK;
    }
    CK(cudaMemcpyAsync(h->d_w, h->d_wt, sizeof(double) * N, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(w_inout, h->d_wt, sizeof(double) * N, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    L.have_prev = true;
    if (alpha_out) *alpha_out = a;
    return ENVAR_OK;
}

// ------------------------------------------------------------------------------------ adjoint loop
// Sec. 3.2 (the paragraph after Eq. gradient_forcing) with the H^1 regularisation of Sec. 4.2.

extern "C" int envar_h1_smooth(envar_handle h, const double *g_dev, double *gs_dev, double l_sob)
{
    if (!h || !g_dev || !gs_dev || !(l_sob >= 0.0)) return ENVAR_EINVAL;
    const int n = h->ncc;
    if (!h->d_h1) { DA(h->d_h1, 3 * (size_t)n); DA(h->d_h1it, 2); }
    for (int comp = 0; comp < 2; ++comp)
        launch_h1_cg(n, h->d_cnb, h->g.dx, h->g.dy, l_sob, g_dev + (size_t)comp * n, gs_dev + (size_t)comp * n, h->d_h1,
                     1e-13, 4 * n + 100, h->d_h1it + comp, h->st);
    int it[2] = {0, 0};
    CK(cudaMemcpyAsync(it, h->d_h1it, sizeof(int) * 2, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    if (it[0] < 0 || it[1] < 0) { set_err(h, "envar_h1_smooth: CG did not converge"); return ENVAR_ESTATE; }
    return ENVAR_OK;
}

// J_obs of one forward run of member slot 0 with control forcing f (device) into *J (host).
static int control_cost(envar_handle h, const double *f, double *J)
{
    launch_compact_to_rect(1, h->nrect, h->ncc, h->d_cidx, f, h->d_frect, h->st);
    if (h->mixed) launch_d2f(2 * (long long)h->nrect, h->d_frect, h->ms.frect, h->st);
    reset_members(h, 1);
    int rc = run_steps(h, 1, h->cfg.n_steps);
    if (rc) return rc;
    enqueue_cost(h, 1, h->d_Jd_slot, h->d_Js_slot, h->d_Yd_slot);
    const double *src = (h->cfg.cost_mode == ENVAR_COST_SENSORS) ? h->d_Js_slot : h->d_Jd_slot;
    MemberCtl c0{};
    CK(cudaMemcpyAsync(J, src, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(&c0, h->d_ctl, sizeof(MemberCtl), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    h->last_member_slot0 = -2;
    if (c0.status) *J = HUGE_VAL;
    return ENVAR_OK;
}

extern "C" int envar_adjoint_lbfgs_reset(envar_handle h, int memory)
{
    if (!h || memory < 1 || memory > 64) return ENVAR_EINVAL;
    return lb_setup(h, h->lbf, h->n_ctrl, memory);
}

extern "C" int envar_adjoint_lbfgs_step(envar_handle h, double *f_inout, int max_snapshots, double l_sob,
                                        double first_step, double *J_out, double *alpha_out, int *evals_out)
{
    if (!h || !f_inout || !(l_sob >= 0.0) || !(first_step > 0.0)) return ENVAR_EINVAL;
    int rc = 0;
    if (h->lbf.m == 0 && (rc = envar_adjoint_lbfgs_reset(h, 8))) return rc;
    LbfgsState &L = h->lbf;
    const int n = h->n_ctrl;
    if (!h->d_fg) { DA(h->d_fg, n); DA(h->d_fgs, n); DA(h->d_fs, n); DA(h->d_dm, 2); }
    // J and dJ/df by the discrete adjoint, the L2 gradient (M_f = dx dy I) and its H^1 smoothing
    double J = 0.0;
    if ((rc = envar_adjoint_gradient(h, f_inout, h->d_fg, max_snapshots, &J))) return rc;
    launch_scale_vec(n, 1.0 / h->g.hxy, h->d_fg, h->d_fs, h->st);
    if ((rc = envar_h1_smooth(h, h->d_fs, h->d_fgs, l_sob))) return rc;
    if ((rc = lb_update(h, L, f_inout, h->d_fgs))) return rc;
    double gp = 0.0, dm[2] = {0.0, 0.0};
    if ((rc = lb_direction(h, L, f_inout, h->d_fgs, 1.0, &gp))) return rc;
    // the Armijo slope is the directional derivative of J itself: dJ/df . p
    launch_dot_max(n, h->d_fg, L.p, h->d_dm, h->st);
    CK(cudaMemcpyAsync(dm, h->d_dm, sizeof(double) * 2, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (!(dm[0] < 0.0)) {
        L.count = 0;
        if ((rc = lb_direction(h, L, f_inout, h->d_fgs, 1.0, &gp))) return rc;
        launch_dot_max(n, h->d_fg, L.p, h->d_dm, h->st);
        CK(cudaMemcpyAsync(dm, h->d_dm, sizeof(double) * 2, cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
    }
    // without curvature pairs the smoothed gradient carries no step length: the first trial moves
    // the control by first_step in the max norm
    double a = (L.count == 0 && dm[1] > 0.0) ? first_step / dm[1] : 1.0;
    const double c1 = 1e-4;
    double Jt = 0.0;
    int evals = 0;
    bool ok = false;
    for (int k = 0; k < 12; ++k) {
        // f_t = f + a p into d_fs
        CK(cudaMemcpyAsync(h->d_fs, f_inout, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
        launch_axpy_vec(n, a, L.p, h->d_fs, h->st);
        if ((rc = control_cost(h, h->d_fs, &Jt))) return rc;
        ++evals;
        ok = Jt <= J + c1 * a * dm[0];
        if (ok) break;
        a *= 0.5;
    }
    h->have_forward = false;
    if (evals_out) *evals_out = evals;
    if (J_out) *J_out = J;
    if (!ok) {
        // no trial decreased J by the Armijo margin: f is stationary to the accuracy of J
        L.have_prev = false;
        if (alpha_out) *alpha_out = 0.0;
        return ENVAR_OK;
    }
    CK(cudaMemcpyAsync(f_inout, h->d_fs, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
    L.have_prev = true;
    if (alpha_out) *alpha_out = a;
    return ENVAR_OK;
}

extern "C" int envar_forward_control(envar_handle h, const double *f, double *J)
{
    if (!h || !f) return ENVAR_EINVAL;
    if (!h->have_ic) { set_err(h, "envar_forward_control: no initial state"); return ENVAR_ESTATE; }
    launch_compact_to_rect(1, h->nrect, h->ncc, h->d_cidx, f, h->d_frect, h->st);
    if (h->mixed) launch_d2f(2 * (long long)h->nrect, h->d_frect, h->ms.frect, h->st);
    reset_members(h, 1);
    int rc = run_steps(h, 1, h->cfg.n_steps);
    if (rc) return rc;
    enqueue_cost(h, 1, h->d_Jd_slot, h->d_Js_slot, h->d_Yd_slot);
    const double *src = (h->cfg.cost_mode == ENVAR_COST_SENSORS) ? h->d_Js_slot : h->d_Jd_slot;
    if (J) CK(cudaMemcpyAsync(J, src, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    h->last_member_slot0 = -2;
    return ENVAR_OK;
}

extern "C" int envar_member_status(envar_handle h, int *status)
{
    if (!h || !status) return ENVAR_EINVAL;
    if (!h->have_forward) { set_err(h, "envar_member_status: no forward run"); return ENVAR_ESTATE; }
    for (int m = 0; m <= h->N; ++m) status[m] = h->ctl_all[m].status;
    return ENVAR_OK;
}

extern "C" int envar_get_state(envar_handle h, int member, double *u, double *v, double *p)
{
    if (!h) return ENVAR_EINVAL;
    int slot = member;
    if (!h->batched) {
        if (member != h->last_member_slot0 && !(member == 0 && h->last_member_slot0 == -2)) {
            set_err(h, "envar_get_state: FP64_PLAIN keeps only the last member run (%d)", h->last_member_slot0);
            return ENVAR_ESTATE;
        }
        slot = 0;
    }
    if (slot < 0 || slot >= h->Mall) return ENVAR_EINVAL;
    const long long off = (long long)slot * h->g.S;
    if (h->mixed)
        launch_export_mx(h->g, h->ms, off, u, v, p, h->st);
    else
        launch_export_state(h->g, h->d_u + off, h->d_v + off, h->d_p + off, u, v, p, h->st);
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    return ENVAR_OK;
}

extern "C" int envar_get_series(envar_handle h, int member, double *series)
{
    if (!h || !series || member < 0 || member > h->N) return ENVAR_EINVAL;
    const int nw = h->cfg.n_window;
    CK(cudaMemcpy(series, h->d_series + (size_t)member * std::max(nw, 1) * 8, sizeof(double) * nw * 8,
                  cudaMemcpyDeviceToHost));
    return ENVAR_OK;
}

extern "C" int envar_diagnostics(envar_handle h, double *max_div, long long *outer_its, long long *inner_its)
{
    if (!h) return ENVAR_EINVAL;
    double md = 0.0;
    long long oi = 0, ii = 0;
    for (const MemberCtl &c : h->ctl_all) {
        md = std::max(md, c.max_div);
        oi += c.outer_its;
        ii += c.inner_its;
    }
    if (max_div) *max_div = md;
    if (outer_its) *outer_its = oi;
    if (inner_its) *inner_its = ii;
    return ENVAR_OK;
}

extern "C" int envar_reset_members(envar_handle h, const double *w)
{
    if (!h) return ENVAR_EINVAL;
    if (!h->have_ic) { set_err(h, "envar_reset_members: no initial state"); return ENVAR_ESTATE; }
    if (h->N > 0 && w) CK(cudaMemcpyAsync(h->d_w, w, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, h->st));
    launch_member_forcing(h->Mall, 0, h->N, h->nrect, h->d_Erect, h->d_w, h->cfg.eps, h->d_frect, h->ms.frect, h->st);
    reset_members(h, h->Mall);
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    h->last_member_slot0 = 0;
    return ENVAR_OK;
}

extern "C" int envar_advance(envar_handle h, int n)
{
    if (!h || n < 0) return ENVAR_EINVAL;
    int rc = run_steps(h, h->Mall, n);
    if (rc) return rc;
    h->ctl_all.assign(h->N + 1, MemberCtl{});
    CK(cudaMemcpyAsync(h->ctl_all.data(), h->d_ctl, sizeof(MemberCtl) * h->Mall, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    return ENVAR_OK;
}

extern "C" int envar_kernel_launches(envar_handle h, long long *count)
{
    (void)h;
    if (!count) return ENVAR_EINVAL;
    *count = launches_so_far() + g_graph_kernels.load() + (long long)conditional_body_launches();
    return ENVAR_OK;
}

extern "C" int envar_time_kernel(envar_handle h, int which, int reps, double *ms)
{
    if (!h || !ms || reps < 1 || which < 0 || which > 8) return ENVAR_EINVAL;
    if (!h->have_ic) { set_err(h, "envar_time_kernel: no initial state"); return ENVAR_ESTATE; }
    const int M = h->Mall;
    std::vector<MemberCtl> c((size_t)M);
    for (int m = 0; m < M; ++m) { c[m] = MemberCtl{}; c[m].step = h->cfg.n_steps; c[m].gidx = h->batched ? m : 0; }
    CK(cudaMemcpyAsync(h->d_ctl, c.data(), sizeof(MemberCtl) * M, cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
    const int wf = h->cfg.cost_mode == ENVAR_COST_DOMAIN ? 1 : 0;
    double *ser = h->cfg.n_window > 0 ? h->d_series_slot : nullptr;
    auto launch = [&]() -> int {
        const Grid &g = h->g;
        switch (which) {
        case 0:
            if (h->mixed)
                launch_predict_rhs_mx(g, h->mc, M, h->ms, h->d_ubc, h->d_inh, h->d_inl, h->d_ctl, h->pt.red,
                                      h->nfluid, h->st);
            else
                launch_predict<double>(g, M, h->d_u, h->d_v, h->d_p, (double *)h->d_Ru, (double *)h->d_Rv, h->d_us,
                                       h->d_vs, h->d_ubc, h->d_frect, h->d_ctl, h->st);
            return 0;
        case 6:
            if (h->mixed) {
                launch_correct_mx(g, h->mc, M, h->ms, h->ms, h->x0, h->y0, wf, ser, h->pt, h->d_ctl, h->cfg.div_tol,
                                  h->nfluid, h->st);
                return 0;
            }
            launch_correct(g, h->x0, h->y0, M, h->d_u, h->d_v, h->d_p, h->d_us, h->d_vs, h->pb.x, h->d_wf, h->d_wd,
                           ref_member(h), wf, ser,
                           h->pt, h->d_ctl, h->cfg.div_tol, h->nfluid, h->st);
            return 0;
        case 8:
            if (h->mixed)
                launch_predict_rhs_mx(g, h->mc, M, h->ms, h->d_ubc, h->d_inh, h->d_inl, h->d_ctl, h->pt.red,
                                      h->nfluid, h->st);
            else launch_rhs(g, M, h->d_us, h->d_vs, h->pb.b, h->d_ctl, h->st);
            return 0;
        default:
            return h->mixed ? launch_poisson_single<float>(which, g, h->lev, M, h->pb, h->pc, h->pt, h->d_ctl, h->st)
                            : launch_poisson_single<double>(which, g, h->lev, M, h->pb, h->pc, h->pt, h->d_ctl, h->st);
        }
    };
    if (launch() != 0) return ENVAR_EINVAL;
    launch();
    // each timed launch starts with a cold L2: a 256 MB write (twice the L2) evicts its inputs
    const size_t flush_bytes = (size_t)256 << 20;
    if (!h->d_flush) DA(h->d_flush, flush_bytes);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double total = 0.0;
    for (int r = 0; r < reps; ++r) {
        CK(cudaMemsetAsync(h->d_flush, r & 0xff, flush_bytes, h->st));
        CK(cudaEventRecord(e0, h->st));
        launch();
        CK(cudaEventRecord(e1, h->st));
        CK(cudaEventSynchronize(e1));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, e0, e1));
        total += t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    *ms = total / reps;
    return ENVAR_OK;
}

extern "C" int envar_apply_preconditioner(envar_handle h, const double *r_dev, double *z_dev)
{
    if (!h || !r_dev || !z_dev) return ENVAR_EINVAL;
    const size_t tsz = h->mixed ? sizeof(float) : sizeof(double);
    CK(cudaMemsetAsync(h->d_ctl, 0, sizeof(MemberCtl) * h->Mall, h->st));
    CK(cudaMemsetAsync(h->pb.r, 0, tsz * (size_t)h->g.S * h->Mall, h->st));
    if (h->mixed) {
        launch_cells_in<float>(h->g, r_dev, (float *)h->pb.r, h->st);
        launch_vcycle<float>(h->g, h->lev, h->Mall, h->pb, h->pc, h->pt, h->d_ctl, h->st);
        launch_cells_out<float>(h->g, (const float *)h->pb.z, z_dev, h->st);
    } else {
        launch_cells_in<double>(h->g, r_dev, (double *)h->pb.r, h->st);
        launch_vcycle<double>(h->g, h->lev, h->Mall, h->pb, h->pc, h->pt, h->d_ctl, h->st);
        launch_cells_out<double>(h->g, (const double *)h->pb.z, z_dev, h->st);
    }
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    return ENVAR_OK;
}

// ------------------------------------------------------------------------------------ adjoint (a9)
// Discrete adjoint of the FP64 stepper for member slot 0 (Sec. 3.2): the kernels are in
// k_adjoint.cu, the checkpoint schedule in revolve.h.  The forward state of a checkpoint is
// (u, v, p, dp, R_u, R_v): the pressure and last increment make a recomputed step bitwise equal
// to the original (the increment is the solve's initial guess), the tendencies carry AB2.
namespace envar {
void launch_adj_rhs(const Grid &g, const double *lu, const double *lv, double *b, unsigned long long *mx,
                    MemberCtl *ctl, cudaStream_t st);
void launch_adj_set_step(MemberCtl *ctl, int k, cudaStream_t st);
void launch_adj_post(const Grid &g, double *lu, double *lv, const double *x, const unsigned long long *mx,
                     const MemberRed *red, double res_tol, MemberCtl *ctl, double *ubb, double *Rbu, double *Rbv,
                     double *cu, double *cv, double *gu, double *gv, double c1, double c0, cudaStream_t st);
void launch_adj_tend(const Grid &g, const double *u, const double *v, const double *Rbu, const double *Rbv,
                     double *lu, double *lv, cudaStream_t st);
void launch_adj_outlet(const Grid &g, const double *ubb, double *lu, cudaStream_t st);
void launch_adj_cost(const Grid &g, const double *u, const double *v, const double *mu, const double *mv, double wgt,
                     double *lu, double *lv, cudaStream_t st);
void launch_faces_to_control(const Grid &g, int ncc, const int *cidx, const double *gu, const double *gv,
                             double *out, cudaStream_t st);
}

static constexpr int kAdjPlanes = 10;          // lu lv cu cv Rbu Rbv gu gv mu mv, then ubb and the scale
static constexpr int kSnapPlanes = 6;          // u v p dp Ru Rv
static constexpr double kAdjResTol = 1e-12;    // max |b - A x| relative to max |b|

struct AdjointExec {
    envar_handle h;
    long long S;
    double *lu, *lv, *cu, *cv, *Rbu, *Rbv, *gu, *gv, *mu, *mv, *ubb;
    unsigned long long *mx;
    int k0;
    double wgt;
    long long cur = -1;   // forward state in the working buffers, -1 if clobbered

    double *plane(int p) const
    {
        switch (p) {
        case 0: return h->d_u;
        case 1: return h->d_v;
        case 2: return h->d_p;
        case 3: return h->pb.x;
        case 4: return (double *)h->d_Ru;
        default: return (double *)h->d_Rv;
        }
    }
    int copy_slot(int slot, bool to_slot)
    {
        double *base = h->d_snap + (size_t)slot * kSnapPlanes * S;
        for (int p = 0; p < kSnapPlanes; ++p) {
            double *w = plane(p), *s = base + (size_t)p * S;
            CK(cudaMemcpyAsync(to_slot ? s : w, to_slot ? w : s, sizeof(double) * S, cudaMemcpyDeviceToDevice, h->st));
        }
        return ENVAR_OK;
    }
    int advance(long long from, long long to)
    {
        int rc = run_steps(h, 1, (int)(to - from));
        if (rc) return rc;
        h->adj_fwd_steps += to - from;
        cur = to;
        return ENVAR_OK;
    }
    int store(int slot, long long k)
    {
        ++h->adj_stores;
        (void)k;
        return copy_slot(slot, true);
    }
    int restore(int slot, long long k)
    {
        if (cur == k) return ENVAR_OK;
        ++h->adj_restores;
        int rc = copy_slot(slot, false);
        if (rc) return rc;
        launch_adj_set_step(h->d_ctl, (int)k, h->st);
        cur = k;
        return ENVAR_OK;
    }
    void enqueue_reverse(bool first, bool in_window)
    {
        const Grid &g = h->g;
        PoissonCfg pa = h->pc;
        pa.rtol_abs = kAdjResTol;
        pa.max_outer = std::max(pa.max_outer, 4);
        launch_adj_rhs(g, lu, lv, h->pb.b, mx, h->d_ctl, h->st);
        cudaMemsetAsync(h->pb.x, 0, sizeof(double) * S, h->st);
        launch_pressure_solve<double>(g, h->lev, 1, h->pb, pa, h->pt, h->d_ctl, h->st);
        launch_adj_post(g, lu, lv, h->pb.x, mx, h->pt.red, kAdjResTol, h->d_ctl, ubb, Rbu, Rbv, cu, cv, gu, gv,
                        first ? 1.0 : 1.5, first ? 0.0 : -0.5, h->st);
        launch_adj_tend(g, h->d_u, h->d_v, Rbu, Rbv, lu, lv, h->st);
        launch_adj_outlet(g, ubb, lu, h->st);
        if (in_window) launch_adj_cost(g, h->d_u, h->d_v, mu, mv, wgt, lu, lv, h->st);
    }
    // reverse step a (a -> a+1) about the working state a, then add the cost gradient at sample a
    int reverse(long long a)
    {
        const int fi = (a == 0) ? 1 : 0, wi = (a >= k0) ? 1 : 0;
        cudaGraphExec_t &ge = h->adj_graph[fi][wi];
        if (!ge) {
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
            set_capturing(true);
            enqueue_reverse(fi != 0, wi != 0);
            set_capturing(false);
            cudaError_t e = cudaStreamEndCapture(h->st, &graph);
            if (e != cudaSuccess || capture_failed()) {
                if (e == cudaSuccess) cudaGraphDestroy(graph);
                set_err(h, "adjoint graph capture failed: %s",
                        e != cudaSuccess ? cudaGetErrorString(e) : "conditional loop body");
                return ENVAR_ECUDA;
            }
            e = cudaGraphInstantiate(&ge, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                ge = nullptr;
                set_err(h, "adjoint graph instantiate failed: %s", cudaGetErrorString(e));
                return ENVAR_ECUDA;
            }
        }
        CK(cudaGraphLaunch(ge, h->st));
        ++h->adj_rev_steps;
        cur = -1;   // the solve used the increment buffer
        return ENVAR_OK;
    }
};

extern "C" int envar_revolve_plan(long long n_steps, int n_slots, long long *recompute, long long *stores,
                                  long long *restores)
{
    if (n_steps < 1 || n_slots < 1) return ENVAR_EINVAL;
    long long st = 0, rs = 0;
    long long f = revolve_dry_run(n_steps, (int)std::min<long long>(n_slots, n_steps), &st, &rs);
    if (f < 0) return ENVAR_ESTATE;
    if (recompute) *recompute = f;
    if (stores) *stores = st;
    if (restores) *restores = rs;
    return ENVAR_OK;
}

extern "C" int envar_adjoint_gradient(envar_handle h, const double *f, double *gf, int max_snapshots, double *J)
{
    if (!h || !f || !gf) return ENVAR_EINVAL;
    if (h->mixed || h->cfg.cost_mode != ENVAR_COST_DOMAIN || h->cfg.n_window < 1 || max_snapshots < 1) {
        set_err(h, "envar_adjoint_gradient: needs an FP64 handle, the DOMAIN cost, n_window >= 1, max_snapshots >= 1");
        return ENVAR_EINVAL;
    }
    if (!h->have_ic) { set_err(h, "envar_adjoint_gradient: no initial state"); return ENVAR_ESTATE; }
    const long long n = h->cfg.n_steps;
    const int Sl = (int)std::min<long long>(max_snapshots, n);
    const long long S = h->g.S;
    if (!h->d_adj) DA(h->d_adj, (size_t)kAdjPlanes * S + h->g.ny + 2);
    if (h->n_snap < Sl) {
        if (h->d_snap) { CK(cudaStreamSynchronize(h->st)); cudaFree(h->d_snap); h->d_snap = nullptr; h->n_snap = 0; }
        void *q = nullptr;
        size_t bytes = sizeof(double) * (size_t)Sl * kSnapPlanes * S;
        cudaError_t e = cudaMalloc(&q, bytes);
        if (e != cudaSuccess) {
            set_err(h, "envar_adjoint_gradient: %d checkpoints need %zu bytes: %s", Sl, bytes, cudaGetErrorString(e));
            return ENVAR_ENOMEM;
        }
        h->d_snap = (double *)q;
        h->n_snap = Sl;
    }
    AdjointExec ex;
    ex.h = h;
    ex.S = S;
    double *a = h->d_adj;
    ex.lu = a; ex.lv = a + S; ex.cu = a + 2 * S; ex.cv = a + 3 * S; ex.Rbu = a + 4 * S; ex.Rbv = a + 5 * S;
    ex.gu = a + 6 * S; ex.gv = a + 7 * S; ex.mu = a + 8 * S; ex.mv = a + 9 * S;
    ex.ubb = a + (size_t)kAdjPlanes * S;
    ex.mx = (unsigned long long *)(ex.ubb + h->g.ny);
    ex.k0 = (int)(n - h->cfg.n_window + 1);
    ex.wgt = h->g.hxy / (double)h->cfg.n_window;
    h->adj_fwd_steps = h->adj_rev_steps = h->adj_stores = h->adj_restores = 0;

    // initial sweep 0 -> n with the forcing f, storing the schedule's first checkpoints
    launch_compact_to_rect(1, h->nrect, h->ncc, h->d_cidx, f, h->d_frect, h->st);
    reset_members(h, 1);
    ex.cur = 0;
    int rc = ex.store(0, 0);
    if (rc) return rc;
    std::vector<long long> pos;
    std::vector<int> slot;
    revolve_spine(n, Sl, &pos, &slot);
    long long at = 0;
    for (size_t k = 0; k < pos.size(); ++k) {
        if ((rc = ex.advance(at, pos[k]))) return rc;
        if ((rc = ex.store(slot[k], pos[k]))) return rc;
        at = pos[k];
    }
    if ((rc = ex.advance(at, n))) return rc;
    enqueue_cost(h, 1, h->d_Jd_slot, h->d_Js_slot, h->d_Yd_slot);
    // window means of the cell-centred velocity (member 0's Welford planes), then lambda^n
    CK(cudaMemcpyAsync(ex.mu, h->d_wf, sizeof(double) * 2 * S, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemsetAsync(a, 0, sizeof(double) * 8 * S, h->st));
    launch_adj_cost(h->g, h->d_u, h->d_v, ex.mu, ex.mv, ex.wgt, ex.lu, ex.lv, h->st);
    if ((rc = revolve_rev(ex, 0, n, Sl - 1, 0, Sl, true))) return rc;
    launch_faces_to_control(h->g, h->ncc, h->d_cidx, ex.gu, ex.gv, gf, h->st);
    MemberCtl c0{};
    CK(cudaMemcpyAsync(&c0, h->d_ctl, sizeof(MemberCtl), cudaMemcpyDeviceToHost, h->st));
    if (J) CK(cudaMemcpyAsync(J, h->d_Jd_slot, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    CK(cudaGetLastError());
    h->have_forward = false;
    h->last_member_slot0 = -2;
    if (c0.status) {
        set_err(h, "envar_adjoint_gradient: status 0x%x (non-finite state, CFL, or an unconverged solve)", c0.status);
        return ENVAR_ESTATE;
    }
    return ENVAR_OK;
}

extern "C" int envar_adjoint_stats(envar_handle h, long long *forward_steps, long long *reverse_steps,
                                   long long *stores, long long *restores)
{
    if (!h) return ENVAR_EINVAL;
    if (forward_steps) *forward_steps = h->adj_fwd_steps;
    if (reverse_steps) *reverse_steps = h->adj_rev_steps;
    if (stores) *stores = h->adj_stores;
    if (restores) *restores = h->adj_restores;
    return ENVAR_OK;
}

// ------------------------------------------------------------------------------------ autotuning
// Solver parameters that change only the speed of a time step (the refinement loop still stops at
// div_tol): refinement cap, inner-iteration cap and tolerance, smoothing sweeps, coarse sweeps.
struct SolverParams { int max_outer, max_inner, nu, coarse_sweeps; double inner_rtol; int nu_coarse; };
// With the refinement loop as a conditional graph node a high refinement cap costs nothing unless
// a step needs it, so every candidate keeps a cap of 10 (margin for the long runs after the probe)
// and the candidates differ in what sets the cost of a refinement.
// The last five smooth the coarser levels less than the finest one (their share of the V-cycle's
// SM time is large and mostly latency).
static const SolverParams kTuneCandidates[] = {
    {10, 2, 3, 2, 1e-3, 0}, {10, 3, 2, 2, 1e-3, 0}, {10, 2, 2, 2, 1e-3, 0}, {10, 3, 3, 2, 1e-3, 0},
    {10, 4, 2, 4, 1e-3, 0}, {10, 2, 3, 4, 1e-3, 0}, {10, 6, 2, 8, 1e-4, 0}, {10, 3, 1, 2, 1e-3, 0},
    {10, 2, 1, 2, 1e-3, 0}, {10, 1, 3, 2, 1e-3, 0}, {10, 1, 2, 2, 1e-3, 0}, {10, 2, 3, 1, 1e-3, 0},
    {10, 2, 3, 1, 1e-3, 1}, {10, 2, 3, 1, 1e-3, 2}, {10, 2, 3, 2, 1e-3, 1}, {10, 3, 3, 1, 1e-3, 1},
    {10, 2, 2, 1, 1e-3, 1},
};

static void drop_graphs(envar_handle h)
{
    for (auto &gs : h->graphs) {
        if (gs.many) cudaGraphExecDestroy(gs.many);
        if (gs.one) cudaGraphExecDestroy(gs.one);
        gs = GraphSet{};
    }
    for (auto &row : h->adj_graph)
        for (auto &ge : row)
            if (ge) { cudaGraphExecDestroy(ge); ge = nullptr; }
}

static void apply_params(envar_handle h, const SolverParams &p)
{
    h->cfg.max_outer = p.max_outer; h->cfg.max_inner = p.max_inner;
    h->cfg.nu_pre = h->cfg.nu_post = p.nu; h->cfg.coarse_sweeps = p.coarse_sweeps; h->cfg.inner_rtol = p.inner_rtol;
    h->cfg.nu_coarse = p.nu_coarse;
    h->pc.max_outer = p.max_outer; h->pc.max_inner = p.max_inner;
    h->pc.nu_pre = h->pc.nu_post = p.nu; h->pc.coarse_sweeps = p.coarse_sweeps; h->pc.nu_c = p.nu_coarse;
    h->pc.inner_rtol2 = p.inner_rtol * p.inner_rtol;
    drop_graphs(h);
}

extern "C" int envar_autotune(envar_handle h, int probe_steps, double *best_ms_per_step, int *chosen)
{
    if (!h || probe_steps < 2) return ENVAR_EINVAL;
    if (!h->have_ic) { set_err(h, "envar_autotune: no initial state"); return ENVAR_ESTATE; }
    const SolverParams orig{h->cfg.max_outer, h->cfg.max_inner, h->cfg.nu_pre, h->cfg.coarse_sweeps, h->cfg.inner_rtol,
                            h->cfg.nu_coarse};
    const int M = h->Mall;
    std::vector<MemberCtl> c((size_t)M);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // on any failure: the original parameters back in place, no event left behind
    auto bail = [&](int rc) {
        apply_params(h, orig);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        h->have_forward = false;
        return rc;
    };
    auto ck = [&](cudaError_t e, const char *what) {
        if (e == cudaSuccess) return ENVAR_OK;
        set_err(h, "envar_autotune: %s failed: %s", what, cudaGetErrorString(e));
        return ENVAR_ECUDA;
    };
    int rc = ck(cudaEventCreate(&e0), "cudaEventCreate");
    if (!rc) rc = ck(cudaEventCreate(&e1), "cudaEventCreate");
    if (rc) return bail(rc);
    double best = -1.0;
    int best_k = -1;
    const int n_cand = (int)(sizeof(kTuneCandidates) / sizeof(kTuneCandidates[0]));
    for (int k = 0; k < n_cand; ++k) {
        apply_params(h, kTuneCandidates[k]);
        // untimed run (captures the graphs), then the timed probe from the same initial state
        float t = 0.f;
        bool ok = true;
        for (int rep = 0; rep < 2 && ok; ++rep) {
            launch_member_forcing(M, 0, h->N, h->nrect, h->d_Erect, h->d_w, h->cfg.eps, h->d_frect, h->ms.frect, h->st);
            reset_members(h, M);
            if ((rc = ck(cudaEventRecord(e0, h->st), "cudaEventRecord"))) return bail(rc);
            if ((rc = run_steps(h, M, probe_steps))) return bail(rc);
            if ((rc = ck(cudaEventRecord(e1, h->st), "cudaEventRecord"))) return bail(rc);
            if ((rc = ck(cudaEventSynchronize(e1), "cudaEventSynchronize"))) return bail(rc);
            if ((rc = ck(cudaEventElapsedTime(&t, e0, e1), "cudaEventElapsedTime"))) return bail(rc);
            if ((rc = ck(cudaMemcpy(c.data(), h->d_ctl, sizeof(MemberCtl) * M, cudaMemcpyDeviceToHost), "cudaMemcpy")))
                return bail(rc);
            for (const MemberCtl &x : c) ok = ok && x.status == 0;
        }
        const double ms = (double)t / probe_steps;
        if (ok && (best < 0 || ms < best)) { best = ms; best_k = k; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    apply_params(h, best_k >= 0 ? kTuneCandidates[best_k] : orig);
    h->have_forward = false;
    h->last_member_slot0 = -2;
    if (best_ms_per_step) *best_ms_per_step = best;
    if (chosen) {
        const SolverParams &p = best_k >= 0 ? kTuneCandidates[best_k] : orig;
        chosen[0] = p.max_outer; chosen[1] = p.max_inner; chosen[2] = p.nu; chosen[3] = p.coarse_sweeps;
    }
    if (best_k < 0) {
        set_err(h, "envar_autotune: no candidate kept every member within div_tol; parameters unchanged");
        return ENVAR_ESTATE;
    }
    return ENVAR_OK;
}

extern "C" int envar_get_config(envar_handle h, envar_config *cfg)
{
    if (!h || !cfg) return ENVAR_EINVAL;
    *cfg = h->cfg;
    return ENVAR_OK;
}
