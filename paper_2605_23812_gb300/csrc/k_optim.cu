// k_optim.cu -- optimisers on the device: the Gauss-Newton Hessian H_GN = Y^T R^{-1} Y + (N-1) I of
// Sec. 3.3.1 (Eq. Hessian_EnVar, R = I) from the sensor-space observation anomalies of Eq. (fdapprox),
// its Cholesky solve for the step dw = -H_GN^{-1} g (Eq. update_Newton), the two-loop recursion of
// the limited-memory BFGS direction (Eq. update_BFGS; in the ensemble weights w or, for the adjoint
// approach of Sec. 3.2, in the control vector f), and the H^1 smoothing of the adjoint gradient of
// Sec. 4.2 (Eq. lsob).
//
// Sizes: N <= 256 perturbations, n_obs = 8 n_window sensor observations, n_ctrl <= 2 x 46 082
// control values.  All of it is small next to one forward run; each kernel is one launch.
#include <algorithm>

#include "envar_internal.cuh"

namespace envar {

// ------------------------------------------------------------------------------ observation anomalies
// Window mean of each (member, channel) of the sensor series [N+1][n_window][8].
__global__ void k_series_means(int nw, const double *__restrict__ series, double *__restrict__ mean)
{
    const int m = blockIdx.x, q = blockIdx.y;
    const double *s = series + (long long)m * nw * 8;
    double acc = 0.0;
    for (int t = threadIdx.x; t < nw; t += blockDim.x) acc += s[(long long)t * 8 + q];
    acc = block_reduce(acc, false);
    if (threadIdx.x == 0) mean[m * 8 + q] = acc / nw;
}

// Y[i][k] = (h_{i+1}[k] - h_0[k]) / eps with h_m = series_m - mean_m (rows of excluded members are 0),
// and h0[k].  k = 8 t + q runs over the n_obs observations.
__global__ void k_sensor_anomalies(int N, int nw, const double *__restrict__ series, const double *__restrict__ mean,
                                   double eps, const int *__restrict__ status, double *__restrict__ Y,
                                   double *__restrict__ h0)
{
    const long long nobs = 8LL * nw;
    const int i = blockIdx.y;   // 0 .. N (row N writes h0)
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nobs; k += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(k & 7);
        const double a0 = series[k] - mean[q];
        if (i == N) {
            h0[k] = a0;
        } else {
            const bool ok = !status || status[i + 1] == 0;
            const double ai = series[(long long)(i + 1) * nobs + k] - mean[(i + 1) * 8 + q];
            Y[(long long)i * nobs + k] = ok ? (ai - a0) / eps : 0.0;
        }
    }
}

void launch_sensor_anomalies(int N, int nw, const double *series, double eps, const int *status, double *mean,
                             double *Y, double *h0, cudaStream_t st)
{
    k_series_means<<<dim3(N + 1, 8), 256, 0, st>>>(nw, series, mean);
    k_sensor_anomalies<<<dim3(cdiv(8 * nw, 256 * 4), N + 1), 256, 0, st>>>(N, nw, series, mean, eps, status, Y, h0);
    count_launches(2);
}

// H[i][j] = Y_i . Y_j + (N-1) delta_ij  (blocks with j >= i; mirrored), and, in the blocks with
// j == N, the gradient g_i = Y_i . h0 + (N-1) w_i of Eq. (gradient_EnVar).  Fixed-order reductions.
__global__ void k_gram(int N, long long nobs, const double *__restrict__ Y, const double *__restrict__ h0,
                       const double *__restrict__ w, double *__restrict__ H, double *__restrict__ g)
{
    const int i = blockIdx.x, j = blockIdx.y;
    if (j < N && j < i) return;
    const double *a = Y + (long long)i * nobs;
    const double *b = (j == N) ? h0 : Y + (long long)j * nobs;
    double acc = 0.0;
    for (long long k = threadIdx.x; k < nobs; k += blockDim.x) acc = fma(a[k], b[k], acc);
    acc = block_reduce(acc, false);
    if (threadIdx.x == 0) {
        if (j == N) {
            g[i] = acc + (double)(N - 1) * w[i];
        } else {
            const double v = acc + (i == j ? (double)(N - 1) : 0.0);
            H[(long long)i * N + j] = v;
            H[(long long)j * N + i] = v;
        }
    }
}

void launch_gram(int N, long long nobs, const double *Y, const double *h0, const double *w, double *H, double *g,
                 cudaStream_t st)
{
    k_gram<<<dim3(N, N + 1), 256, 0, st>>>(N, nobs, Y, h0, w, H, g);
    count_launches(1);
}

// ------------------------------------------------------------------------------ Cholesky solve
// One block: L L^T = A (A: N x N SPD, row-major, copied to the work matrix Lw), then
// w_out = w - alpha A^{-1} g.  *info = 0, or j + 1 if the j-th pivot is not positive (w_out
// untouched).  Right-looking: per column one pivot, the column scaled, the trailing block updated.
__global__ void __launch_bounds__(1024) k_cholesky_step(int N, const double *__restrict__ A, double *__restrict__ Lw,
                                                        const double *__restrict__ g, const double *__restrict__ w,
                                                        double alpha, double *__restrict__ x, double *__restrict__ w_out,
                                                        int *info)
{
    __shared__ double s_piv;
    __shared__ int s_bad;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (long long q = tid; q < (long long)N * N; q += nt) Lw[q] = A[q];
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int j = 0; j < N; ++j) {
        if (tid == 0) {
            const double d = Lw[(long long)j * N + j];
            if (!(d > 0.0)) s_bad = j + 1;
            s_piv = (d > 0.0) ? sqrt(d) : 1.0;
            Lw[(long long)j * N + j] = s_piv;
        }
        __syncthreads();
        if (s_bad) break;
        const double piv = s_piv;
        for (int i = j + 1 + tid; i < N; i += nt) Lw[(long long)i * N + j] /= piv;
        __syncthreads();
        // trailing update A[i][k] -= L[i][j] L[k][j], k <= i
        const int m = N - j - 1;
        for (long long q = tid; q < (long long)m * m; q += nt) {
            const int i = j + 1 + (int)(q / m), k = j + 1 + (int)(q % m);
            if (k <= i) Lw[(long long)i * N + k] -= Lw[(long long)i * N + j] * Lw[(long long)k * N + j];
        }
        __syncthreads();
    }
    if (s_bad) {
        if (tid == 0) *info = s_bad;
        return;
    }
    // forward and back substitution (serial in one warp's lane 0: N <= 256 rows)
    if (tid == 0) {
        for (int i = 0; i < N; ++i) {
            double a = g[i];
            for (int k = 0; k < i; ++k) a -= Lw[(long long)i * N + k] * x[k];
            x[i] = a / Lw[(long long)i * N + i];
        }
        for (int i = N - 1; i >= 0; --i) {
            double a = x[i];
            for (int k = i + 1; k < N; ++k) a -= Lw[(long long)k * N + i] * x[k];
            x[i] = a / Lw[(long long)i * N + i];
        }
        for (int i = 0; i < N; ++i) w_out[i] = w[i] - alpha * x[i];
        *info = 0;
    }
}

void launch_cholesky_step(int N, const double *A, double *Lw, const double *g, const double *w, double alpha, double *x,
                          double *w_out, int *info, cudaStream_t st)
{
    k_cholesky_step<<<1, 1024, 0, st>>>(N, A, Lw, g, w, alpha, x, w_out, info);
    count_launches(1);
}

// ------------------------------------------------------------------------------ L-BFGS
// Store the pair s = w - w_prev, y = g - g_prev in ring slot `slot` ([m][N] arrays) and its
// curvature s^T y in sy[slot]; also |s|^2 |y|^2 in sy[m + slot] for the acceptance test.
__global__ void k_lbfgs_pair(int N, const double *__restrict__ w, const double *__restrict__ wp,
                             const double *__restrict__ g, const double *__restrict__ gp, int slot,
                             double *__restrict__ S, double *__restrict__ Yh, double *__restrict__ sy, int m)
{
    double a = 0.0, ss = 0.0, yy = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double s = w[i] - wp[i], y = g[i] - gp[i];
        S[(long long)slot * N + i] = s;
        Yh[(long long)slot * N + i] = y;
        a += s * y;
        ss += s * s;
        yy += y * y;
    }
    a = block_reduce(a, false);
    ss = block_reduce(ss, false);
    yy = block_reduce(yy, false);
    if (threadIdx.x == 0) {
        sy[slot] = a;
        sy[m + slot] = ss * yy;
    }
}

void launch_lbfgs_pair(int N, const double *w, const double *wp, const double *g, const double *gp, int slot,
                       double *S, double *Yh, double *sy, int m, cudaStream_t st)
{
    k_lbfgs_pair<<<1, 256, 0, st>>>(N, w, wp, g, gp, slot, S, Yh, sy, m);
    count_launches(1);
}

// Two-loop recursion over the `count` stored pairs, newest first then oldest first, with the
// ring's slots in age order order[0] (oldest) .. order[count-1] (newest); H0 = gamma I with
// gamma = s^T y / y^T y of the newest pair, or gamma0 without pairs.  p = -H g, and gp = g^T p.
__global__ void k_lbfgs_direction(int N, int count, const int *__restrict__ order, const double *__restrict__ S,
                                  const double *__restrict__ Yh, const double *__restrict__ g, double gamma0,
                                  double *__restrict__ q, double *__restrict__ alpha, double *__restrict__ p,
                                  double *__restrict__ gp)
{
    for (int i = threadIdx.x; i < N; i += blockDim.x) q[i] = g[i];
    __syncthreads();
    for (int r = count - 1; r >= 0; --r) {
        const double *s = S + (long long)order[r] * N, *y = Yh + (long long)order[r] * N;
        double sy = 0.0, sq = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) { sy += s[i] * y[i]; sq += s[i] * q[i]; }
        sy = block_reduce(sy, false);
        sq = block_reduce(sq, false);
        const double a = sq / sy;
        if (threadIdx.x == 0) alpha[r] = a;
        for (int i = threadIdx.x; i < N; i += blockDim.x) q[i] -= a * y[i];
        __syncthreads();
    }
    double gamma = gamma0;
    if (count > 0) {
        const double *s = S + (long long)order[count - 1] * N, *y = Yh + (long long)order[count - 1] * N;
        double sy = 0.0, yy = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) { sy += s[i] * y[i]; yy += y[i] * y[i]; }
        sy = block_reduce(sy, false);
        yy = block_reduce(yy, false);
        gamma = sy / yy;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) q[i] *= gamma;
    __syncthreads();
    for (int r = 0; r < count; ++r) {
        const double *s = S + (long long)order[r] * N, *y = Yh + (long long)order[r] * N;
        double sy = 0.0, yq = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) { sy += s[i] * y[i]; yq += y[i] * q[i]; }
        sy = block_reduce(sy, false);
        yq = block_reduce(yq, false);
        const double b = yq / sy;
        const double a = alpha[r];
        for (int i = threadIdx.x; i < N; i += blockDim.x) q[i] += s[i] * (a - b);
        __syncthreads();
    }
    double d = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        p[i] = -q[i];
        d -= g[i] * q[i];
    }
    d = block_reduce(d, false);
    if (threadIdx.x == 0) *gp = d;
}

void launch_lbfgs_direction(int N, int count, const int *order, const double *S, const double *Yh, const double *g,
                            double gamma0, double *q, double *alpha, double *p, double *gp, cudaStream_t st)
{
    k_lbfgs_direction<<<1, 256, 0, st>>>(N, count, order, S, Yh, g, gamma0, q, alpha, p, gp);
    count_launches(1);
}

// w_t = w + a p, and (N-1)/2 w_t^T w_t (the prior part of Eq. J_w at the trial point).
__global__ void k_trial_point(int N, const double *__restrict__ w, const double *__restrict__ p, double a,
                              double *__restrict__ wt, double *__restrict__ prior)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double v = w[i] + a * p[i];
        wt[i] = v;
        acc += v * v;
    }
    acc = block_reduce(acc, false);
    if (threadIdx.x == 0) *prior = 0.5 * (double)(N - 1) * acc;
}

void launch_trial_point(int N, const double *w, const double *p, double a, double *wt, double *prior, cudaStream_t st)
{
    k_trial_point<<<1, 256, 0, st>>>(N, w, p, a, wt, prior);
    count_launches(1);
}

} // namespace envar

namespace envar {

// ------------------------------------------------------------------------------ H^1 smoothing
// Eq. (lsob): (I - l^2 Lap) x = (1 + l^2) g on the n control cells of one forcing component, Lap
// the 5-point Laplacian with no flux through the boundary of the control set (nb[4][n]: the E, W,
// N, S neighbour control cell or -1).  Conjugate gradients in one block (the operator is SPD, with
// condition number at most 1 + 8 l^2 / h^2), until |r| <= rtol |b| or max_it iterations; *iters
// receives the iterations, negative if the tolerance was not met.
__device__ __forceinline__ double h1_apply(int q, const double *__restrict__ x, const int *__restrict__ nb, int n,
                                           double cxl, double cyl)
{
    const double xq = x[q];
    double lap = 0.0;
    const int e = nb[q], w = nb[n + q], no = nb[2 * n + q], so = nb[3 * n + q];
    if (e >= 0) lap += cxl * (x[e] - xq);
    if (w >= 0) lap += cxl * (x[w] - xq);
    if (no >= 0) lap += cyl * (x[no] - xq);
    if (so >= 0) lap += cyl * (x[so] - xq);
    return xq - lap;
}

__global__ void __launch_bounds__(1024) k_h1_cg(int n, const int *__restrict__ nb, double cxl, double cyl, double scale,
                                                const double *__restrict__ g, double *__restrict__ x,
                                                double *__restrict__ r, double *__restrict__ p, double *__restrict__ Ap,
                                                double rtol, int max_it, int *iters)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    double bb = 0.0;
    for (int q = tid; q < n; q += nt) {
        const double b = scale * g[q];
        x[q] = 0.0;
        r[q] = b;
        p[q] = b;
        bb += b * b;
    }
    bb = block_reduce(bb, false);
    double rr = bb;
    int it = 0;
    bool done = !(bb > 0.0);
    while (!done && it < max_it) {
        double pAp = 0.0;
        for (int q = tid; q < n; q += nt) {
            const double a = h1_apply(q, p, nb, n, cxl, cyl);
            Ap[q] = a;
            pAp += p[q] * a;
        }
        pAp = block_reduce(pAp, false);
        const double alpha = rr / pAp;
        double rr1 = 0.0;
        for (int q = tid; q < n; q += nt) {
            x[q] += alpha * p[q];
            r[q] -= alpha * Ap[q];
            rr1 += r[q] * r[q];
        }
        rr1 = block_reduce(rr1, false);
        ++it;
        done = rr1 <= rtol * rtol * bb;
        const double beta = rr1 / rr;
        rr = rr1;
        if (!done)
            for (int q = tid; q < n; q += nt) p[q] = r[q] + beta * p[q];
        __syncthreads();
    }
    if (tid == 0) *iters = done ? it : -it;
}

void launch_h1_cg(int n, const int *nb, double dx, double dy, double l_sob, const double *g, double *x, double *work,
                  double rtol, int max_it, int *iters, cudaStream_t st)
{
    const double l2 = l_sob * l_sob;
    k_h1_cg<<<1, 1024, 0, st>>>(n, nb, l2 / (dx * dx), l2 / (dy * dy), 1.0 + l2, g, x, work, work + n, work + 2 * n,
                               rtol, max_it, iters);
    count_launches(1);
}

// y = a x (elementwise scale), and the directional derivative d = g^T p of two n-vectors.
__global__ void k_scale_vec(long long n, double a, const double *__restrict__ x, double *__restrict__ y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = a * x[i];
}
void launch_scale_vec(long long n, double a, const double *x, double *y, cudaStream_t st)
{
    const int grid = (int)std::min<long long>((n + 255) / 256, 1024);
    k_scale_vec<<<grid, 256, 0, st>>>(n, a, x, y);
    count_launches(1);
}

// y += a x
__global__ void k_axpy_vec(long long n, double a, const double *__restrict__ x, double *__restrict__ y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}
void launch_axpy_vec(long long n, double a, const double *x, double *y, cudaStream_t st)
{
    const int grid = (int)std::min<long long>((n + 255) / 256, 1024);
    k_axpy_vec<<<grid, 256, 0, st>>>(n, a, x, y);
    count_launches(1);
}

__global__ void k_dot_max(long long n, const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ out)
{
    double d = 0.0, m = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        d += a[i] * b[i];
        m = fmax(m, fabs(b[i]));
    }
    d = block_reduce(d, false);
    m = block_reduce(m, true);
    if (threadIdx.x == 0) { out[0] = d; out[1] = m; }
}
void launch_dot_max(long long n, const double *a, const double *b, double *out, cudaStream_t st)
{
    k_dot_max<<<1, 1024, 0, st>>>(n, a, b, out);
    count_launches(1);
}

} // namespace envar
