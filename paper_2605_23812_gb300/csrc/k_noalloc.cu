// k_noalloc.cu -- ensemble draw without any device allocation.
//
// envar_init allocates its buffers with cudaMalloc.  Some callers cannot let a library allocate
// device memory at all: a framework whose caching allocator owns the whole device and forbids
// foreign cudaMalloc/cudaFree calls, an embedding that runs with a fixed memory budget, or code
// that must not trigger the synchronisation a cudaFree implies.  For them,
// envar_draw_ensemble_noalloc draws the same ensemble matrix E as envar_init + envar_get_ensemble,
// writing it straight into a caller-owned buffer and using, as scratch, a file-scope __device__
// array of fixed size (ENVAR_NOALLOC_SCRATCH_BYTES) that every GPU which loads this library
// holds until the process exits.
//
// Set-up: the first call on a device, with that device current, looks the array's device address
// up once (cudaGetSymbolAddress; host code cannot use the symbol itself as a device pointer) and
// caches it per device.  Make that first call before any stream capture.
// The scratch is shared by all calls: calls that overlap on the GPU (different streams or
// threads) race on it.  Every scratch element a call reads is written earlier in the same call,
// so the contents left by a previous call never matter.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <vector>

#include "envar_internal.cuh"
#include "../../include/envar.h"

namespace envar {
void launch_axis_factor(double h, double a, int ncell, int m, int pad, int nxi, double *G, cudaStream_t st);
void set_global_error(const char *msg);
}
using namespace envar;

static __device__ __align__(256) unsigned char g_noalloc_scratch[ENVAR_NOALLOC_SCRATCH_BYTES];

static constexpr int kMaxDevices = 64;
static void *g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mu;
// failures are reported through envar_last_error(NULL)
static int fail(int rc, const char *msg, cudaError_t e = cudaSuccess)
{
    char buf[256];
    if (e != cudaSuccess)
        std::snprintf(buf, sizeof(buf), "envar_draw_ensemble_noalloc: %s: %s", msg, cudaGetErrorString(e));
    else
        std::snprintf(buf, sizeof(buf), "envar_draw_ensemble_noalloc: %s", msg);
    set_global_error(buf);
    return rc;
}

static int scratch_base(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(ENVAR_ECUDA, "cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) return fail(ENVAR_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return fail(ENVAR_ECUDA, "cudaGetSymbolAddress(scratch)", e);
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return ENVAR_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

extern "C" int envar_draw_ensemble_noalloc(const envar_config *cfg, double *E_dev, int n_ctrl, void *cuda_stream)
{
    if (!cfg || !E_dev) return fail(ENVAR_EINVAL, "null argument");
    // a launch error left behind by unrelated earlier work on this thread is not this call's
    (void)cudaGetLastError();
    const envar_config &c = *cfg;
    if (c.nx < 8 || c.ny < 4 || c.n_members < 1 || !(c.corr_len > 0) || !(c.x1 > c.x0) || !(c.y1 > c.y0))
        return fail(ENVAR_EINVAL, "invalid configuration");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nx = c.nx, ny = c.ny, N = c.n_members;
    const double dx = (c.x1 - c.x0) / nx, dy = (c.y1 - c.y0) / ny;
    // control rectangle and control cells (host): same rule as envar_init
    int ia = -1, ib = -1, ja = -1, jb = -1;
    for (int i = 0; i < nx; ++i) {
        double x = c.x0 + ((double)i + 0.5) * dx;
        if (x >= c.region[0] && x <= c.region[1]) { if (ia < 0) ia = i; ib = i; }
    }
    for (int j = 0; j < ny; ++j) {
        double y = c.y0 + ((double)j + 0.5) * dy;
        if (y >= c.region[2] && y <= c.region[3]) { if (ja < 0) ja = j; jb = j; }
    }
    if (ia < 0 || ja < 0) return fail(ENVAR_EINVAL, "control region contains no cell centre");
    const int nrx = ib - ia + 1, nry = jb - ja + 1, nrect = nrx * nry;
    std::vector<int> cidx;
    std::vector<uint8_t> rc((size_t)nrect, 0);
    for (int j = ja; j <= jb; ++j)
        for (int i = ia; i <= ib; ++i) {
            double x = c.x0 + ((double)i + 0.5) * dx, y = c.y0 + ((double)j + 0.5) * dy;
            if ((y > 0.0) || (x > 0.0 && x < 1.0)) {
                int r = (j - ja) * nrx + (i - ia);
                cidx.push_back(r);
                rc[r] = 1;
            }
        }
    const int ncc = (int)cidx.size();
    // lattice sizes (same as envar_init)
    auto axis = [&](double hh, int ncell, int *m, int *pad, int *nxi) {
        int mm = (int)std::ceil(4.0 * hh / c.corr_len);
        if (mm < 1) mm = 1;
        *m = mm;
        *pad = (int)std::ceil(5.0 * c.corr_len / (hh / mm));
        *nxi = (ncell - 1) * mm + 1 + 2 * (*pad);
    };
    int mx, px, nxix, my, py, nxiy;
    axis(dx, nrx, &mx, &px, &nxix);
    axis(dy, nry, &my, &py, &nxiy);
    // scratch plan (one member at a time): Gx, Gy, Z, T, Erect (double), cidx (int), rect mask
    const size_t bGx = align256(sizeof(double) * (size_t)nrx * nxix), bGy = align256(sizeof(double) * (size_t)nry * nxiy);
    const size_t bZ = align256(sizeof(double) * 2 * (size_t)nxiy * nxix), bT = align256(sizeof(double) * 2 * (size_t)nxiy * nrx);
    const size_t bE = align256(sizeof(double) * 2 * (size_t)nrect), bC = align256(sizeof(int) * (size_t)ncc);
    const size_t bR = align256((size_t)nrect);
    const size_t need = bGx + bGy + bZ + bT + bE + bC + bR;
    if (need > (size_t)ENVAR_NOALLOC_SCRATCH_BYTES)
        return fail(ENVAR_EINVAL, "configuration needs more scratch than ENVAR_NOALLOC_SCRATCH_BYTES (8 MiB)");
    if (n_ctrl != 2 * ncc) return fail(ENVAR_EINVAL, "n_ctrl does not match the control region");
    void *base = nullptr;
    int rcode = scratch_base(&base);
    if (rcode) return rcode;
    char *p = (char *)base;
    double *Gx = (double *)p; p += bGx;
    double *Gy = (double *)p; p += bGy;
    double *Z = (double *)p; p += bZ;
    double *T = (double *)p; p += bT;
    double *Er = (double *)p; p += bE;
    int *dc = (int *)p; p += bC;
    uint8_t *dr = (uint8_t *)p;
    cudaError_t e = cudaMemcpyAsync(dc, cidx.data(), sizeof(int) * ncc, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dr, rc.data(), (size_t)nrect, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(ENVAR_ECUDA, "cudaMemcpyAsync", e);
    launch_axis_factor(dx, c.corr_len, nrx, mx, px, nxix, Gx, st);
    launch_axis_factor(dy, c.corr_len, nry, my, py, nxiy, Gy, st);
    const long long per_member = 2LL * nxiy * nxix;
    for (int k = 0; k < N; ++k) {
        launch_normals(c.seed, 0ULL, (long long)k * per_member, per_member, Z, st);
        launch_conv_sampler(1, nrx, nry, nxix, nxiy, Gx, Gy, Z, dr, c.sigma, Er, T, st);
        launch_rect_to_compact(1, nrect, ncc, dc, Er, E_dev + (size_t)k * n_ctrl, st);
    }
    if (c.forcing_y_only) {   // zero prior variance on the fx entries, as envar_init does
        e = cudaMemset2DAsync(E_dev, sizeof(double) * n_ctrl, 0, sizeof(double) * ncc, N, st);
        if (e != cudaSuccess) return fail(ENVAR_ECUDA, "cudaMemset2DAsync", e);
    }
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) return fail(ENVAR_ECUDA, "ensemble draw launch", e);
    // the host vectors above are read by the copies: wait for them before returning
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(ENVAR_ECUDA, "ensemble draw", e);
    return ENVAR_OK;
}
