// GMRES-IR rung of the mixed-precision solver: outer refinement whose
// correction equation A d = r is solved by restarted flexible GMRES
// (Saad 1993) with the FP32 LU factors as right preconditioner
// (z = U^{-1} L^{-1} P v computed in FP32) and FP64 products with A
// (Carson and Higham 2017 analyse this GMRES-IR scheme; the flexible variant
// keeps the Arnoldi relation exact in FP64 whatever the preconditioner error).
// Orthogonalisation: classical Gram-Schmidt applied twice.  The small
// Hessenberg least-squares problem is solved on the host with Givens rotations.
#include "common.cuh"
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace lu {
int solve_f32_perm(int n, int nrhs, const float *LU, int lda, const int *perm, float *B, int ldb, cudaStream_t s);
cudaError_t launch_residual(int n, int nrhs, const double *A, int lda, const double *X, int ldx, const double *B, int ldb,
                            double *R, int ldr, double *part, unsigned long long *rmax, cudaStream_t s);
size_t residual_workspace_doubles(int n, int nrhs);
cudaError_t launch_absmax(int n, int nrhs, const double *V, int ldv, unsigned long long *out, cudaStream_t s);

constexpr int kDotThreads = 512;

// out[c] = sum_i V[i, c] * w[i] for c < ncols, one CTA per column (fixed order)
__global__ void dots_kernel(int n, int ncols, const double *__restrict__ V, int ldv, const double *__restrict__ w,
                            double *__restrict__ out) {
    __shared__ double red[kDotThreads / 32];
    const int c = blockIdx.x;
    if (c >= ncols) return;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kDotThreads) s = fma(V[(size_t)i + (size_t)c * ldv], w[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < kDotThreads / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) out[c] = s;
    }
}

// w := w - V[:, 0:ncols] h   (h on the device)
__global__ void sub_vh_kernel(int n, int ncols, const double *__restrict__ V, int ldv, const double *__restrict__ h,
                              double *__restrict__ w) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double acc = w[i];
        for (int c = 0; c < ncols; ++c) acc = fma(-V[(size_t)i + (size_t)c * ldv], h[c], acc);
        w[i] = acc;
    }
}

// y := a * x (FP64), or into FP32
__global__ void scale_kernel(int n, double a, const double *__restrict__ x, double *__restrict__ y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = a * x[i];
}
__global__ void to_f32_kernel(int n, const double *__restrict__ x, float *__restrict__ y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = (float)x[i];
}
__global__ void to_f64_kernel(int n, const float *__restrict__ x, double *__restrict__ y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = (double)x[i];
}
// x += Z y (y on the device, k entries)
__global__ void add_zy_kernel(int n, int k, const double *__restrict__ Z, int ldz, const double *__restrict__ y,
                              double *__restrict__ x) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < k; ++c) acc = fma(Z[(size_t)i + (size_t)c * ldz], y[c], acc);
        x[i] += acc;
    }
}

static int g1(int n) { return std::min(lu_ceil_div(n, 256), 152 * 8); }

static double b2d(unsigned long long b) {
    double d;
    memcpy(&d, &b, sizeof(d));
    return d;
}

// FGMRES-IR on each right-hand side column.  On return X holds the refined
// solution and *eta_out the worst backward error.
int gmres_ir(int n, int nrhs, const double *A, int lda, const double *B, int ldb, double *X, int ldx, const float *LU32,
             int ld32, const int *perm, double anorm, const double *bnorm, double tol, int max_outer, int restart,
             int *iters_out, int *inner_out, double *eta_out, cudaStream_t s) {
    const int m = std::max(1, restart);
    double *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr, *part = nullptr, *dv = nullptr;
    float *t32 = nullptr;
    unsigned long long *nrm = nullptr;
    LU_CUDA_TRY(cudaMallocAsync(&V, sizeof(double) * (size_t)n * (m + 1), s));
    LU_CUDA_TRY(cudaMallocAsync(&Z, sizeof(double) * (size_t)n * m, s));
    LU_CUDA_TRY(cudaMallocAsync(&w, sizeof(double) * n, s));
    LU_CUDA_TRY(cudaMallocAsync(&r, sizeof(double) * n, s));
    LU_CUDA_TRY(cudaMallocAsync(&part, sizeof(double) * residual_workspace_doubles(n, 1), s));
    LU_CUDA_TRY(cudaMallocAsync(&dv, sizeof(double) * (m + 2), s));
    LU_CUDA_TRY(cudaMallocAsync(&t32, sizeof(float) * n, s));
    LU_CUDA_TRY(cudaMallocAsync(&nrm, sizeof(unsigned long long) * 2, s));
    int outer_total = 0, inner_total = 0;
    double worst = 0.0;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), h(m + 1), y(m);
    for (int q = 0; q < nrhs; ++q) {
        double *x = X + (size_t)q * ldx;
        const double *b = B + (size_t)q * ldb;
        double eta = INFINITY;
        std::vector<double> hist;
        for (int outer = 0; outer <= max_outer; ++outer) {
            // r = b - A x and its backward error
            LU_CUDA_TRY(launch_residual(n, 1, A, lda, x, n, b, n, r, n, part, nrm, s));
            LU_CUDA_TRY(launch_absmax(n, 1, x, n, nrm + 1, s));
            unsigned long long hn[2];
            LU_CUDA_TRY(cudaMemcpyAsync(hn, nrm, sizeof(hn), cudaMemcpyDeviceToHost, s));
            LU_CUDA_TRY(cudaStreamSynchronize(s));
            const double den = anorm * b2d(hn[1]) + bnorm[q];
            eta = den > 0 ? b2d(hn[0]) / den : 0.0;
            if (std::isnan(eta)) eta = INFINITY;
            hist.push_back(eta);
            if (eta <= tol || outer == max_outer) break;
            const size_t hs = hist.size();
            if (hs >= 3 && !(hist[hs - 1] <= 0.5 * hist[hs - 3])) break;   // stalled
            ++outer_total;
            // beta = ||r||_2, v_0 = r / beta
            double beta = 0.0;
            dots_kernel<<<1, kDotThreads, 0, s>>>(n, 1, r, n, r, dv);
            lu_count_launch();
            LU_CUDA_TRY(cudaMemcpyAsync(&beta, dv, sizeof(double), cudaMemcpyDeviceToHost, s));
            LU_CUDA_TRY(cudaStreamSynchronize(s));
            beta = std::sqrt(beta);
            if (!(beta > 0.0) || !std::isfinite(beta)) break;
            scale_kernel<<<g1(n), 256, 0, s>>>(n, 1.0 / beta, r, V);
            lu_count_launch();
            std::fill(g.begin(), g.end(), 0.0);
            g[0] = beta;
            int k = 0;
            for (int j = 0; j < m; ++j) {
                // z_j = M^{-1} v_j in FP32, kept in FP64
                to_f32_kernel<<<g1(n), 256, 0, s>>>(n, V + (size_t)j * n, t32);
                lu_count_launch();
                int rc = solve_f32_perm(n, 1, LU32, ld32, perm, t32, n, s);
                if (rc != LU_OK) return rc;
                to_f64_kernel<<<g1(n), 256, 0, s>>>(n, t32, Z + (size_t)j * n);
                lu_count_launch();
                // w = A z_j  (FP64)
                LU_CUDA_TRY(launch_residual(n, 1, A, lda, Z + (size_t)j * n, n, nullptr, n, w, n, part, nrm, s));
                // classical Gram-Schmidt, twice
                std::fill(h.begin(), h.end(), 0.0);
                for (int pass = 0; pass < 2; ++pass) {
                    dots_kernel<<<j + 1, kDotThreads, 0, s>>>(n, j + 1, V, n, w, dv);
                    lu_count_launch();
                    sub_vh_kernel<<<g1(n), 256, 0, s>>>(n, j + 1, V, n, dv, w);
                    lu_count_launch();
                    std::vector<double> hp(j + 1);
                    LU_CUDA_TRY(cudaMemcpyAsync(hp.data(), dv, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s));
                    LU_CUDA_TRY(cudaStreamSynchronize(s));
                    for (int i = 0; i <= j; ++i) h[i] += hp[i];
                }
                dots_kernel<<<1, kDotThreads, 0, s>>>(n, 1, w, n, w, dv);
                lu_count_launch();
                double hn2 = 0.0;
                LU_CUDA_TRY(cudaMemcpyAsync(&hn2, dv, sizeof(double), cudaMemcpyDeviceToHost, s));
                LU_CUDA_TRY(cudaStreamSynchronize(s));
                h[j + 1] = std::sqrt(hn2);
                if (h[j + 1] > 0.0) {
                    scale_kernel<<<g1(n), 256, 0, s>>>(n, 1.0 / h[j + 1], w, V + (size_t)(j + 1) * n);
                    lu_count_launch();
                }
                // apply previous rotations, then a new one to zero h[j+1]
                for (int i = 0; i < j; ++i) {
                    const double t = cs[i] * h[i] + sn[i] * h[i + 1];
                    h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
                    h[i] = t;
                }
                const double den2 = std::hypot(h[j], h[j + 1]);
                cs[j] = den2 > 0 ? h[j] / den2 : 1.0;
                sn[j] = den2 > 0 ? h[j + 1] / den2 : 0.0;
                h[j] = den2;
                h[j + 1] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h[i];
                k = j + 1;
                ++inner_total;
                if (std::fabs(g[j + 1]) <= 1e-10 * beta || hn2 == 0.0) break;
            }
            // y = R^{-1} g (upper triangular back substitution)
            for (int i = k - 1; i >= 0; --i) {
                double t = g[i];
                for (int c = i + 1; c < k; ++c) t -= H[(size_t)i * m + c] * y[c];
                y[i] = H[(size_t)i * m + i] != 0.0 ? t / H[(size_t)i * m + i] : 0.0;
            }
            LU_CUDA_TRY(cudaMemcpyAsync(dv, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
            add_zy_kernel<<<g1(n), 256, 0, s>>>(n, k, Z, n, dv, x);
            lu_count_launch();
            LU_CUDA_TRY(cudaStreamSynchronize(s));   // y is a host buffer reused next cycle
        }
        worst = std::max(worst, eta);
    }
    cudaFreeAsync(V, s);
    cudaFreeAsync(Z, s);
    cudaFreeAsync(w, s);
    cudaFreeAsync(r, s);
    cudaFreeAsync(part, s);
    cudaFreeAsync(dv, s);
    cudaFreeAsync(t32, s);
    cudaFreeAsync(nrm, s);
    LU_CUDA_TRY(cudaGetLastError());
    *iters_out = outer_total;
    *inner_out = inner_total;
    *eta_out = worst;
    return LU_OK;
}

}  // namespace lu
