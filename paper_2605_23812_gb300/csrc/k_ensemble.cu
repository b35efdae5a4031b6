// k_ensemble.cu -- ensemble generation, member forcings and the EnVar projection (Sec. 3.3).
//
//  * normals: Philox4x64-10 (Salmon et al., SC'11) of counter (q/4, 0, 0, 0) and key (seed, stream),
//    two Box-Muller pairs per block of four 64-bit words.
//  * conv sampler: columns of E are draws from N(0, B), B_ij = sigma^2 exp(-|x_i - x_j|^2 / a^2)
//    (Eq. covarianceB with a_x = a_y = a, c_xy = infinity), computed as sigma (Gx (x) Gy) Z with white
//    noise Z on a lattice of spacing <= a/4 and G[r][k] = c exp(-2 (x_r - xi_k)^2 / a^2): the lattice
//    sum of G G^T reproduces the Gaussian kernel to rounding, with no ill-conditioned factorisation.
//  * member forcing: f_m = E w + eps E_m (Eq. ensemble_representation with f_e = 0; Eq. fdapprox).
//  * gradients: g = Y^T (Hq_0 - y) + (N-1) w (Eq. gradient_EnVar) with Y from Eq. (fdapprox), either
//    on the sensor series (exact contraction) or through the scalar cost anomalies.
#include "envar_internal.cuh"

namespace envar {

__device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0, unsigned long long k1)
{
    const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        unsigned long long n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
}

__global__ void k_normals(unsigned long long seed, unsigned long long stream, long long first, long long n,
                          double *__restrict__ out)
{
    const double two_m53 = 1.0 / 9007199254740992.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        long long q = first + t;
        unsigned long long c[4] = {(unsigned long long)(q / 4), 0ULL, 0ULL, 0ULL};
        philox4x64_10(c, seed, stream);
        int lane = (int)(q % 4);
        unsigned long long a = (lane < 2) ? c[0] : c[2], b = (lane < 2) ? c[1] : c[3];
        double u1 = ((double)(a >> 11) + 1.0) * two_m53;
        double u2 = (double)(b >> 11) * two_m53;
        double rad = sqrt(-2.0 * log(u1));
        double s, co;
        sincospi(2.0 * u2, &s, &co);
        out[t] = (lane % 2 == 0) ? rad * co : rad * s;
    }
}

void launch_normals(unsigned long long seed, unsigned long long stream, long long first, long long n, double *out,
                    cudaStream_t st)
{
    if (n <= 0) return;
    long long nb = (n + 255) / 256;
    k_normals<<<(unsigned)(nb < 65535 ? nb : 65535), 256, 0, st>>>(seed, stream, first, n, out);
    count_launches(1);
}

// 1-D factor G[r][k] = c exp(-2 (x_r - xi_k)^2 / a^2) on the lattice xi_k = x_first + (k - pad) eta.
__global__ void k_axis_factor(double h, double a, int ncell, int m, int pad, int nxi, double *__restrict__ G)
{
    const double eta = h / m;
    const double c = sqrt(2.0 * eta / (a * sqrt(3.14159265358979323846)));
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ncell * nxi; t += gridDim.x * blockDim.x) {
        int r = t / nxi, k = t % nxi;
        double d = (double)r * h - (double)(k - pad) * eta;
        G[t] = c * exp(-2.0 * d * d / (a * a));
    }
}

void launch_axis_factor(double h, double a, int ncell, int m, int pad, int nxi, double *G, cudaStream_t st)
{
    int n = ncell * nxi;
    k_axis_factor<<<(n + 255) / 256, 256, 0, st>>>(h, a, ncell, m, pad, nxi, G);
    count_launches(1);
}

// T[k][c][ky][ix] = sum_kx Gx[ix][kx] Z[k][c][ky][kx]
__global__ void k_contract_x(int NC, int nrx, int nxix, int nxiy, const double *__restrict__ Gx,
                             const double *__restrict__ Z, double *__restrict__ T)
{
    long long n = (long long)NC * nxiy * nrx;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        int ix = (int)(t % nrx);
        long long kcy = t / nrx;              // (k*2+c)*nxiy + ky
        const double *z = Z + kcy * nxix;
        const double *gx = Gx + (long long)ix * nxix;
        double acc = 0.0;
        for (int kx = 0; kx < nxix; ++kx) acc += gx[kx] * z[kx];
        T[t] = acc;
    }
}

// Erect[k][c][iy][ix] = sigma * sum_ky Gy[iy][ky] T[k][c][ky][ix]   (zero outside control cells)
__global__ void k_contract_y(int NC, int nrx, int nry, int nxiy, const double *__restrict__ Gy,
                             const double *__restrict__ T, const uint8_t *__restrict__ rect_ctrl, double sigma,
                             double *__restrict__ E)
{
    long long n = (long long)NC * nry * nrx;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        int ix = (int)(t % nrx);
        int iy = (int)((t / nrx) % nry);
        long long kc = t / ((long long)nrx * nry);
        double acc = 0.0;
        if (rect_ctrl[iy * nrx + ix]) {
            const double *tt = T + kc * nxiy * nrx + ix;
            const double *gy = Gy + (long long)iy * nxiy;
            for (int ky = 0; ky < nxiy; ++ky) acc += gy[ky] * tt[(long long)ky * nrx];
        }
        E[t] = sigma * acc;
    }
}

void launch_conv_sampler(int N, int nrx, int nry, int nxix, int nxiy, const double *Gx, const double *Gy,
                         const double *Z, const uint8_t *rect_ctrl, double sigma, double *Erect, double *tmp,
                         cudaStream_t st)
{
    int NC = 2 * N;
    long long n1 = (long long)NC * nxiy * nrx, n2 = (long long)NC * nry * nrx;
    k_contract_x<<<(unsigned)((n1 + 255) / 256 < 65535 ? (n1 + 255) / 256 : 65535), 256, 0, st>>>(NC, nrx, nxix, nxiy,
                                                                                                   Gx, Z, tmp);
    k_contract_y<<<(unsigned)((n2 + 255) / 256 < 65535 ? (n2 + 255) / 256 : 65535), 256, 0, st>>>(
        NC, nrx, nry, nxiy, Gy, tmp, rect_ctrl, sigma, Erect);
    count_launches(2);
}

// f[m][c][rect] = sum_k E[k][c][rect] w_k + (member > 0 ? eps E[member-1][c][rect] : 0)
__global__ void k_member_forcing(int M, int first_member, int N, int nrect, const double *__restrict__ E,
                                 const double *__restrict__ w, double eps, double *__restrict__ f,
                                 float *__restrict__ ff)
{
    long long n = (long long)M * 2 * nrect;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        int r = (int)(t % (2LL * nrect));      // c * nrect + cell
        int slot = (int)(t / (2LL * nrect));
        int member = first_member + slot;
        double acc = 0.0;
        for (int k = 0; k < N; ++k) acc += E[(long long)k * 2 * nrect + r] * w[k];
        if (member > 0) acc += eps * E[(long long)(member - 1) * 2 * nrect + r];
        f[t] = acc;
        if (ff) ff[t] = (float)acc;
    }
}

void launch_member_forcing(int M, int first_member, int N, int nrect, const double *Erect, const double *w,
                           double eps, double *frect, float *frect_f, cudaStream_t st)
{
    long long n = (long long)M * 2 * nrect;
    k_member_forcing<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(M, first_member, N, nrect, Erect, w, eps, frect,
                                                                  frect_f);
    count_launches(1);
}

__global__ void k_scatter(int N, int nrect, int ncc, const int *__restrict__ cidx, const double *__restrict__ E,
                          double *__restrict__ Erect)
{
    long long n = (long long)N * 2 * ncc;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        int q = (int)(t % ncc);
        long long kc = t / ncc;   // k*2 + c
        Erect[kc * nrect + cidx[q]] = E[t];
    }
}
__global__ void k_gather(int N, int nrect, int ncc, const int *__restrict__ cidx, const double *__restrict__ Erect,
                         double *__restrict__ E)
{
    long long n = (long long)N * 2 * ncc;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        int q = (int)(t % ncc);
        long long kc = t / ncc;
        E[t] = Erect[kc * nrect + cidx[q]];
    }
}

void launch_compact_to_rect(int N, int nrect, int ncc, const int *cidx, const double *E, double *Erect, cudaStream_t st)
{
    cudaMemsetAsync(Erect, 0, sizeof(double) * (size_t)N * 2 * nrect, st);
    long long n = (long long)N * 2 * ncc;
    if (n > 0) k_scatter<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(N, nrect, ncc, cidx, E, Erect);
    count_launches(1);
}
void launch_rect_to_compact(int N, int nrect, int ncc, const int *cidx, const double *Erect, double *E, cudaStream_t st)
{
    long long n = (long long)N * 2 * ncc;
    if (n > 0) k_gather<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(N, nrect, ncc, cidx, Erect, E);
    count_launches(1);
}

// ---------------------------------------------------------------- gradients (K9)
// Scalar-anomaly form: g_i = (J_i - J_0)/eps + (N-1) w_i;  J_prior = (N-1)/2 w^T w.
// Scalar-anomaly form: g_i = (J_i - J_0)/eps + (N-1) w_i, also J_prior = (N-1)/2 w^T w (Eq. J_w).
// A member with a nonzero status word keeps only the prior term.
__global__ void k_scalar_gradient(int N, const double *__restrict__ J, const double *__restrict__ w, double eps,
                                  const int *__restrict__ status, double *__restrict__ g, double *__restrict__ jprior)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const bool ok = !status || status[i + 1] == 0;
        g[i] = (ok ? (J[i + 1] - J[0]) / eps : 0.0) + (double)(N - 1) * w[i];
        acc += w[i] * w[i];
    }
    acc = block_reduce(acc, false);
    if (threadIdx.x == 0 && jprior) *jprior = 0.5 * (double)(N - 1) * acc;
}

void launch_scalar_gradient(int N, const double *J, const double *w, double eps, const int *status, double *g,
                            double *jprior, cudaStream_t st)
{
    k_scalar_gradient<<<1, 256, 0, st>>>(N, J, w, eps, status, g, jprior);
    count_launches(1);
}

// DOMAIN form of Eq. (gradient_EnVar) with Y_i = (h_i - h_0)/eps from Eq. (fdapprox):
//   Y_i^T h_0 = (1/2||h_i||^2 - 1/2||h_0||^2 - 1/2||h_i - h_0||^2) / eps = (J_i - J_0 - Yd_i)/eps,
// with Yd_i = 1/2||h_i - h_0||^2 accumulated in the correction kernel (Welford of u_i - u_0).
__global__ void k_domain_gradient(int N, const double *__restrict__ J, const double *__restrict__ Yd,
                                  const double *__restrict__ w, double eps, const int *__restrict__ status,
                                  double *__restrict__ g)
{
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const bool ok = !status || status[i + 1] == 0;
        g[i] = (ok ? (J[i + 1] - J[0] - Yd[i + 1]) / eps : 0.0) + (double)(N - 1) * w[i];
    }
}

void launch_domain_gradient(int N, const double *J, const double *Yd, const double *w, double eps, const int *status,
                            double *g, cudaStream_t st)
{
    k_domain_gradient<<<1, 256, 0, st>>>(N, J, Yd, w, eps, status, g);
    count_launches(1);
}

// Sensor form: h_m(t,s) = series_m(t,s) - mean_t series_m(., s);  Y_i = (h_i - h_0)/eps;
// g_i = Y_i^T h_0 + (N-1) w_i.  One block per i.
__global__ void k_sensor_gradient(int N, int nw, const double *__restrict__ series, double eps,
                                  const double *__restrict__ w, const int *__restrict__ status,
                                  double *__restrict__ g)
{
    const int i = blockIdx.x;
    const double *s0 = series;
    const double *si = series + (long long)(i + 1) * nw * 8;
    double acc = 0.0;
    for (int q = 0; q < 8; ++q) {
        double m0 = 0.0, mi = 0.0;
        for (int t = threadIdx.x; t < nw; t += blockDim.x) {
            m0 += s0[(long long)t * 8 + q];
            mi += si[(long long)t * 8 + q];
        }
        m0 = block_reduce(m0, false) / nw;
        mi = block_reduce(mi, false) / nw;
        double a = 0.0;
        for (int t = threadIdx.x; t < nw; t += blockDim.x) {
            double h0 = s0[(long long)t * 8 + q] - m0, hi = si[(long long)t * 8 + q] - mi;
            a += (hi - h0) / eps * h0;
        }
        acc += block_reduce(a, false);
    }
    const bool ok = !status || status[i + 1] == 0;
    if (threadIdx.x == 0) g[i] = (ok ? acc : 0.0) + (double)(N - 1) * w[i];
}

void launch_sensor_gradient(int N, int n_window, const double *series, double eps, const double *w,
                            const int *status, double *g, cudaStream_t st)
{
    if (N > 0) k_sensor_gradient<<<N, 256, 0, st>>>(N, n_window, series, eps, w, status, g);
    count_launches(1);
}

// df = scale * E g   (E compact n_ctrl x N column-major)
__global__ void k_df(int N, int n_ctrl, const double *__restrict__ E, const double *__restrict__ g, double scale,
                     double *__restrict__ df)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_ctrl; r += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < N; ++k) acc += E[(long long)k * n_ctrl + r] * g[k];
        df[r] = scale * acc;
    }
}
void launch_df(int N, int n_ctrl, const double *E, const double *g, double scale, double *df, cudaStream_t st)
{
    k_df<<<(n_ctrl + 255) / 256, 256, 0, st>>>(N, n_ctrl, E, g, scale, df);
    count_launches(1);
}

__global__ void k_total_cost(const double *J, const double *jp, double *out) { *out = J[0] + *jp; }
void launch_total_cost(const double *J, const double *jp, double *out, cudaStream_t st)
{
    k_total_cost<<<1, 1, 0, st>>>(J, jp, out);
    count_launches(1);
}

__global__ void k_d2f(long long n, const double *__restrict__ a, float *__restrict__ b)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        b[t] = (float)a[t];
}
void launch_d2f(long long n, const double *a, float *b, cudaStream_t st)
{
    if (n <= 0) return;
    k_d2f<<<(unsigned)((n + 255) / 256 < 65535 ? (n + 255) / 256 : 65535), 256, 0, st>>>(n, a, b);
    count_launches(1);
}

// compact [ny][nx] <-> padded level-0 cell layout (one member slot)
template <class TM>
__global__ void k_cells_in(int nx, int ny, int P, const double *__restrict__ src, TM *__restrict__ dst)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i < nx) dst[(long long)j * P + i] = (TM)src[(long long)j * nx + i];
}
template <class TM>
__global__ void k_cells_out(int nx, int ny, int P, const TM *__restrict__ src, double *__restrict__ dst)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i < nx) dst[(long long)j * nx + i] = (double)src[(long long)j * P + i];
}
template <class TM>
void launch_cells_in(const Grid &g, const double *src, TM *dst, cudaStream_t st)
{
    k_cells_in<TM><<<dim3(cdiv(g.nx, 128), g.ny), 128, 0, st>>>(g.nx, g.ny, g.P, src, dst);
    count_launches(1);
}
template <class TM>
void launch_cells_out(const Grid &g, const TM *src, double *dst, cudaStream_t st)
{
    k_cells_out<TM><<<dim3(cdiv(g.nx, 128), g.ny), 128, 0, st>>>(g.nx, g.ny, g.P, src, dst);
    count_launches(1);
}
template void launch_cells_in<float>(const Grid &, const double *, float *, cudaStream_t);
template void launch_cells_in<double>(const Grid &, const double *, double *, cudaStream_t);
template void launch_cells_out<float>(const Grid &, const float *, double *, cudaStream_t);
template void launch_cells_out<double>(const Grid &, const double *, double *, cudaStream_t);

__global__ void k_update_w(int N, double *w, const double *g, double step)
{
    for (int i = threadIdx.x; i < N; i += blockDim.x) w[i] -= step * g[i];
}
void launch_update_w(int N, double *w, const double *g, double step, cudaStream_t st)
{
    k_update_w<<<1, 256, 0, st>>>(N, w, g, step);
    count_launches(1);
}

} // namespace envar
