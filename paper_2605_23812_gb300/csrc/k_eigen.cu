// k_eigen.cu -- the eigenvector ensemble of Sec. 3.3.2 (Eq. eigenvm1) on the device:
//   B = U Sigma U^T, U^T M_f U = I,  E = U_N Sigma_N^{1/2} sqrt(N - 1).
// On the uniform control cells M_f = dx dy I cancels, so E = V_N Lambda_N^{1/2} sqrt(N - 1) with
// (V, Lambda) the Euclidean eigenpairs of the one-component covariance B_s (Eq. covarianceB with
// c_xy = infinity) restricted to the control cells; both forcing components share B_s, so every
// eigenvector of B_s gives one fx and one fy member.
//
// B_s x = sigma^2 gather( K_y scatter(x) K_x ) with the 1-D Gaussian kernels K_x (nrx x nrx) and
// K_y (nry x nry) of the control rectangle: B_s is never formed.  Its leading eigenpairs come from
// Lanczos with full reorthogonalisation (two classical Gram-Schmidt passes per step), the
// tridiagonal projection is diagonalised by parallel cyclic Jacobi in one block, and the Ritz
// vectors are Q S.  All of this runs once per ensemble, before any forward run.
#include <algorithm>
#include <vector>

#include "envar_internal.cuh"

namespace envar {

// K[i][j] = exp(-((i - j) h)^2 / a^2)
__global__ void k_gauss_kernel(int n, double h, double a, double *__restrict__ K)
{
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)n * n) return;
    const int i = (int)(q / n), j = (int)(q % n);
    const double d = (i - j) * h;
    K[q] = exp(-d * d / (a * a));
}

// C[M x N] = A[M x K] B[K x N], row-major FP64, 16 x 16 shared-memory tiles.
__global__ void k_gemm_nn(int M, int N, int K, const double *__restrict__ A, const double *__restrict__ B,
                          double *__restrict__ C)
{
    __shared__ double sa[16][17], sb[16][17];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
    double acc = 0.0;
    for (int k0 = 0; k0 < K; k0 += 16) {
        sa[ty][tx] = (row < M && k0 + tx < K) ? A[(long long)row * K + k0 + tx] : 0.0;
        sb[ty][tx] = (k0 + ty < K && col < N) ? B[(long long)(k0 + ty) * N + col] : 0.0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = fma(sa[ty][k], sb[k][tx], acc);
        __syncthreads();
    }
    if (row < M && col < N) C[(long long)row * N + col] = acc;
}

static void gemm_nn(int M, int N, int K, const double *A, const double *B, double *C, cudaStream_t st)
{
    dim3 blk(16, 16), grd(cdiv(N, 16), cdiv(M, 16));
    k_gemm_nn<<<grd, blk, 0, st>>>(M, N, K, A, B, C);
    count_launches(1);
}

__global__ void k_scatter_cc(int ncc, const int *__restrict__ cidx, const double *__restrict__ x,
                             double *__restrict__ R)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < ncc) R[cidx[q]] = x[q];
}
__global__ void k_gather_cc(int ncc, const int *__restrict__ cidx, const double *__restrict__ R, double scale,
                            double *__restrict__ y)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < ncc) y[q] = scale * R[cidx[q]];
}

// c[k] = Q_k . w for the rows k = 0 .. nq-1 of Q ([rows][n]); with nq + 1 blocks the last block
// also gives |w|^2 into c[nq].
__global__ void k_dots(int n, int nq, const double *__restrict__ Q, const double *__restrict__ w, double *__restrict__ c)
{
    const int k = blockIdx.x;
    const double *a = (k < nq) ? Q + (long long)k * n : w;
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc = fma(a[i], w[i], acc);
    acc = block_reduce(acc, false);
    if (threadIdx.x == 0) c[k] = acc;
}

// w -= sum_k c[k] Q_k, and acc[k] += c[k] (the projection coefficients of both passes)
__global__ void k_subtract(int n, int nq, const double *__restrict__ Q, const double *__restrict__ c,
                           double *__restrict__ w)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = w[i];
    for (int k = 0; k < nq; ++k) v -= c[k] * Q[(long long)k * n + i];
    w[i] = v;
}

// T[j][j] = c1[j] + c2[j]; beta = |w| (from c2[nq]); q_{j+1} = w / beta; T[j][j+1] = T[j+1][j] = beta
__global__ void k_lanczos_close(int n, int j, int m, const double *__restrict__ c1, const double *__restrict__ c2,
                                const double *__restrict__ w, double *__restrict__ qnext, double *__restrict__ T,
                                double *__restrict__ beta_out)
{
    const double beta = sqrt(fmax(c2[j + 1], 0.0));
    const double inv = (beta > 0.0) ? 1.0 / beta : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) qnext[i] = w[i] * inv;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        T[(long long)j * m + j] = c1[j] + c2[j];
        if (j + 1 < m) {
            T[(long long)j * m + j + 1] = beta;
            T[(long long)(j + 1) * m + j] = beta;
        }
        beta_out[j] = beta;
    }
}

__global__ void k_normalize(int n, double *__restrict__ q)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += q[i] * q[i];
    acc = block_reduce(acc, false);
    const double inv = 1.0 / sqrt(acc);
    for (int i = threadIdx.x; i < n; i += blockDim.x) q[i] *= inv;
}

// Parallel cyclic Jacobi on the symmetric m x m matrix A (m even; row-major, in place) with the
// circle ordering: in round r of a sweep, element m-1 meets r and element (r + k) meets (r - k),
// both mod m-1, so the m/2 rotations of a round act on disjoint index pairs.  V accumulates the
// rotations (A_in = V diag(A_out) V^T).  Stops when the off-diagonal Frobenius norm falls below
// tol times the full norm, or after max_sweeps sweeps; *sweeps_out receives the sweeps used.
__global__ void __launch_bounds__(1024) k_jacobi(int m, double *__restrict__ A, double *__restrict__ V, double tol,
                                                 int max_sweeps, int *sweeps_out)
{
    extern __shared__ double sh[];   // c[m/2], s[m/2], then pairs p[m/2], q[m/2] as ints
    double *cs = sh, *sn = sh + m / 2;
    int *pp = reinterpret_cast<int *>(sn + m / 2), *qq = pp + m / 2;
    const int tid = threadIdx.x, nt = blockDim.x, h = m / 2;
    for (long long e = tid; e < (long long)m * m; e += nt) V[e] = ((e / m) == (e % m)) ? 1.0 : 0.0;
    __syncthreads();
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        double off = 0.0, all = 0.0;
        for (long long e = tid; e < (long long)m * m; e += nt) {
            const double a = A[e];
            all += a * a;
            if ((e / m) != (e % m)) off += a * a;
        }
        off = block_reduce(off, false);
        all = block_reduce(all, false);
        if (off <= tol * tol * all) break;
        for (int r = 0; r < m - 1; ++r) {
            for (int k = tid; k < h; k += nt) {
                int p, q;
                if (k == 0) { p = r; q = m - 1; }
                else { p = (r + k) % (m - 1); q = (r - k + (m - 1)) % (m - 1); }
                if (p > q) { const int t = p; p = q; q = t; }
                const double apq = A[(long long)p * m + q];
                double c = 1.0, s = 0.0;
                if (apq != 0.0) {
                    const double tau = (A[(long long)q * m + q] - A[(long long)p * m + p]) / (2.0 * apq);
                    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + t * t);
                    s = t * c;
                }
                cs[k] = c; sn[k] = s; pp[k] = p; qq[k] = q;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (long long e = tid; e < (long long)h * m; e += nt) {
                const int k = (int)(e / m), j = (int)(e % m);
                const int p = pp[k], q = qq[k];
                const double c = cs[k], s = sn[k];
                const double ap = A[(long long)p * m + j], aq = A[(long long)q * m + j];
                A[(long long)p * m + j] = c * ap - s * aq;
                A[(long long)q * m + j] = s * ap + c * aq;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (long long e = tid; e < (long long)h * m; e += nt) {
                const int k = (int)(e / m), i = (int)(e % m);
                const int p = pp[k], q = qq[k];
                const double c = cs[k], s = sn[k];
                const double ap = A[(long long)i * m + p], aq = A[(long long)i * m + q];
                A[(long long)i * m + p] = c * ap - s * aq;
                A[(long long)i * m + q] = s * ap + c * aq;
                const double vp = V[(long long)i * m + p], vq = V[(long long)i * m + q];
                V[(long long)i * m + p] = c * vp - s * vq;
                V[(long long)i * m + q] = s * vp + c * vq;
            }
            __syncthreads();
        }
    }
    if (tid == 0) *sweeps_out = sweep;
}

// Indices of the k largest diagonal entries of A (m x m), in decreasing order (one thread; m small).
__global__ void k_top_diag(int m, int k, const double *__restrict__ A, int *__restrict__ idx, double *__restrict__ lam)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int r = 0; r < k; ++r) {
        int best = -1;
        for (int i = 0; i < m; ++i) {
            bool used = false;
            for (int t = 0; t < r; ++t) used |= (idx[t] == i);
            if (used) continue;
            if (best < 0 || A[(long long)i * m + i] > A[(long long)best * m + best]) best = i;
        }
        idx[r] = best;
        lam[r] = A[(long long)best * m + best];
    }
}

// Sk[r][j] = S[j][idx[r]]: the eigenvector coefficients of the k kept Ritz pairs, as rows.
__global__ void k_gather_ritz(int m, int k, const double *__restrict__ S, const int *__restrict__ idx,
                              double *__restrict__ Sk)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * k) return;
    const int r = e / m, j = e % m;
    Sk[e] = S[(long long)j * m + idx[r]];
}

// Ritz vector r (row r of v = Sk Q): normalised, sign so that its largest-magnitude entry is
// positive, scaled by sqrt(lambda_r (N-1)); written as members 2r (fx) and 2r+1 (fy) of E
// (n_ctrl x N column-major, zero elsewhere), when those members exist, or, with y_only, as the fy
// member r.  One block per r.
__global__ void k_ritz_members(int n, int N, int y_only, const double *__restrict__ lam, const double *__restrict__ v,
                               double *__restrict__ E)
{
    const int r = blockIdx.x;
    const double *vr = v + (long long)r * n;
    double nrm = 0.0, amax = -1.0;
    int imax = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double a = vr[i];
        nrm += a * a;
        if (fabs(a) > amax) { amax = fabs(a); imax = i; }
    }
    nrm = block_reduce(nrm, false);
    // arg-max |v| (ties: lowest index) through the shared-memory reduction of block_reduce's layout
    __shared__ double s_val[1024];
    __shared__ int s_idx[1024];
    s_val[threadIdx.x] = amax;
    s_idx[threadIdx.x] = imax;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double a = s_val[threadIdx.x + o];
            const int ia = s_idx[threadIdx.x + o];
            if (a > s_val[threadIdx.x] || (a == s_val[threadIdx.x] && ia < s_idx[threadIdx.x])) {
                s_val[threadIdx.x] = a;
                s_idx[threadIdx.x] = ia;
            }
        }
        __syncthreads();
    }
    const double sgn = (vr[s_idx[0]] < 0.0) ? -1.0 : 1.0;
    const double scale = sgn * sqrt(fmax(lam[r], 0.0) * (double)(N - 1)) / sqrt(nrm);
    const long long nctrl = 2LL * n;
    for (int comp = y_only ? 1 : 0; comp < 2; ++comp) {
        const int k = y_only ? r : 2 * r + comp;
        if (k >= N) break;
        double *Ek = E + (long long)k * nctrl;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            Ek[(long long)comp * n + i] = scale * vr[i];
            Ek[(long long)(1 - comp) * n + i] = 0.0;
        }
    }
}

// Residual bound of the k kept Ritz pairs after m Lanczos steps: |B v_r - theta_r v_r| =
// beta_m |S[m-1][idx_r]| (exact in exact arithmetic; with full reorthogonalisation a faithful
// estimate).  bound[r] = that / theta_1.
__global__ void k_ritz_bounds(int m, int k, const double *__restrict__ S, const int *__restrict__ idx,
                              const double *__restrict__ lam, double beta, double *__restrict__ bound)
{
    const int r = threadIdx.x;
    if (r < k) bound[r] = fabs(beta * S[(long long)(m - 1) * m + idx[r]]) / fmax(lam[0], 1e-300);
}

// copy the leading m x m block of T (stored with row length mmax) to A (row length m)
__global__ void k_copy_block(int m, int mmax, const double *__restrict__ T, double *__restrict__ A)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e < (long long)m * m) A[e] = T[(e / m) * mmax + (e % m)];
}

size_t eigen_work_doubles(int nrx, int nry, int ncc, int mmax, int k)
{
    return (size_t)nrx * nrx + (size_t)nry * nry + 2 * (size_t)nrx * nry + (size_t)(mmax + 1) * ncc + ncc +
           2 * (size_t)(mmax + 2) + 3 * (size_t)mmax * mmax + mmax + 2 * (size_t)k + (size_t)k * ncc +
           (size_t)k * mmax + (size_t)k + 8;
}

// Leading k eigenpairs of B_s by Lanczos; writes the N members of E (compact, column-major).  The
// Lanczos basis grows from m0 steps, doubling up to mmax (<= ncc), until every kept Ritz pair's
// residual bound is below tol times the largest eigenvalue.  work: eigen_work_doubles(..., mmax, k)
// doubles.  Host outputs (nullable): the k eigenvalues, the steps used, the largest bound.
int eigen_ensemble(int nrx, int nry, double dx, double dy, double a, double sigma, int ncc, const int *cidx, int N,
                   int y_only, int m0, int mmax, double tol, unsigned long long seed, double *work, double *E,
                   double *lam_host, int *steps_host, double *bound_host, cudaStream_t st)
{
    const int k = y_only ? N : (N + 1) / 2;
    mmax -= mmax % 2;
    m0 = std::min(m0 - m0 % 2, mmax);
    if (m0 < 2 || k > m0) return -1;
    double *p = work;
    double *Kx = p; p += (size_t)nrx * nrx;
    double *Ky = p; p += (size_t)nry * nry;
    double *R = p; p += (size_t)nrx * nry;
    double *T1 = p; p += (size_t)nrx * nry;
    double *Q = p; p += (size_t)(mmax + 1) * ncc;
    double *w = p; p += ncc;
    double *c1 = p; p += mmax + 2;
    double *c2 = p; p += mmax + 2;
    double *T = p; p += (size_t)mmax * mmax;
    double *A = p; p += (size_t)mmax * mmax;
    double *V = p; p += (size_t)mmax * mmax;
    double *beta = p; p += mmax;
    double *lam = p; p += k;
    double *bound = p; p += k;
    double *vr = p; p += (size_t)k * ncc;
    double *Sk = p; p += (size_t)k * mmax;
    int *idx = reinterpret_cast<int *>(p); p += k;
    int *sweeps = reinterpret_cast<int *>(p);

    k_gauss_kernel<<<cdiv(nrx * nrx, 256), 256, 0, st>>>(nrx, dx, a, Kx);
    k_gauss_kernel<<<cdiv(nry * nry, 256), 256, 0, st>>>(nry, dy, a, Ky);
    count_launches(2);
    cudaMemsetAsync(T, 0, sizeof(double) * (size_t)mmax * mmax, st);
    launch_normals(seed, 7ULL, 0LL, ncc, Q, st);   // seeded start vector
    k_normalize<<<1, 1024, 0, st>>>(ncc, Q);
    count_launches(1);
    const int gb = cdiv(ncc, 256);
    int done = 0, m = m0;
    std::vector<double> hb((size_t)k);
    double worst = 0.0;
    for (;;) {
        for (int j = done; j < m; ++j) {
            const double *qj = Q + (size_t)j * ncc;
            // w = B_s q_j
            cudaMemsetAsync(R, 0, sizeof(double) * (size_t)nrx * nry, st);
            k_scatter_cc<<<gb, 256, 0, st>>>(ncc, cidx, qj, R);
            count_launches(1);
            gemm_nn(nry, nrx, nry, Ky, R, T1, st);
            gemm_nn(nry, nrx, nrx, T1, Kx, R, st);
            k_gather_cc<<<gb, 256, 0, st>>>(ncc, cidx, R, sigma * sigma, w);
            // two Gram-Schmidt passes against q_0 .. q_j, then |w|^2 into c2[j+1]
            k_dots<<<j + 1, 256, 0, st>>>(ncc, j + 1, Q, w, c1);
            k_subtract<<<gb, 256, 0, st>>>(ncc, j + 1, Q, c1, w);
            k_dots<<<j + 1, 256, 0, st>>>(ncc, j + 1, Q, w, c2);
            k_subtract<<<gb, 256, 0, st>>>(ncc, j + 1, Q, c2, w);
            k_dots<<<1, 256, 0, st>>>(ncc, 0, Q, w, c2 + j + 1);
            k_lanczos_close<<<gb, 256, 0, st>>>(ncc, j, mmax, c1, c2, w, Q + (size_t)(j + 1) * ncc, T, beta);
            count_launches(7);
        }
        done = m;
        const size_t smem = sizeof(double) * m + sizeof(int) * m;
        k_copy_block<<<cdiv(m * m, 256), 256, 0, st>>>(m, mmax, T, A);
        k_jacobi<<<1, 1024, smem, st>>>(m, A, V, 1e-15, 60, sweeps);
        k_top_diag<<<1, 32, 0, st>>>(m, k, A, idx, lam);
        count_launches(3);
        double bm = 0.0;
        cudaMemcpyAsync(&bm, beta + (m - 1), sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        k_ritz_bounds<<<1, 256, 0, st>>>(m, k, V, idx, lam, bm, bound);
        count_launches(1);
        cudaMemcpyAsync(hb.data(), bound, sizeof(double) * k, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        worst = 0.0;
        for (double b : hb) worst = std::max(worst, b);
        if (worst <= tol || m >= mmax) break;
        m = std::min(2 * m, mmax);
    }
    k_gather_ritz<<<cdiv(m * k, 256), 256, 0, st>>>(m, k, V, idx, Sk);
    count_launches(1);
    gemm_nn(k, ncc, m, Sk, Q, vr, st);
    k_ritz_members<<<k, 1024, 0, st>>>(ncc, N, y_only, lam, vr, E);
    count_launches(1);
    if (lam_host) cudaMemcpyAsync(lam_host, lam, sizeof(double) * k, cudaMemcpyDeviceToHost, st);
    if (steps_host) *steps_host = m;
    if (bound_host) *bound_host = worst;
    return 0;
}

} // namespace envar
