// GMRES-IR rung of the mixed-precision solver: outer refinement whose
// correction equation A d = r is solved by restarted flexible GMRES
// (Saad 1993) with the FP32 LU factors as right preconditioner
// (z = U^{-1} L^{-1} P v computed in FP32) and FP64 products with A
// (Carson and Higham 2017 analyse this GMRES-IR scheme; the flexible variant
// keeps the Arnoldi relation exact in FP64 whatever the preconditioner error).
// Orthogonalisation: classical Gram-Schmidt applied twice.  The small
// Hessenberg least-squares problem is solved on the host with Givens rotations.
// The right-hand side columns run side by side, up to kGmresChunk at a time:
// each keeps its own Krylov basis, Hessenberg matrix and stopping decisions,
// while one multi-column preconditioner solve, one multi-column product with
// A and one host synchronisation per Gram-Schmidt pass serve all of them.
#include "common.cuh"
#include "internal.h"
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

namespace lu {

constexpr int kDotThreads = 512;
constexpr int kGmresChunk = 16;   // right-hand side columns iterated together

// Column q of a family: base + q * stride.  out[q * ostride + c] = V_q[:, c] . w_q
// for c < ncols; grid (ncols, Q), one CTA per dot product (fixed order).
__global__ void dots_kernel(int n, int ncols, const double *__restrict__ V, size_t vstride, int ldv,
                            const double *__restrict__ w, size_t wstride, double *__restrict__ out, int ostride) {
    __shared__ double red[kDotThreads / 32];
    const int c = blockIdx.x, q = blockIdx.y;
    if (c >= ncols) return;
    const double *v = V + (size_t)q * vstride + (size_t)c * ldv;
    const double *x = w + (size_t)q * wstride;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kDotThreads) s = fma(v[i], x[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < kDotThreads / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) out[(size_t)q * ostride + c] = s;
    }
}

// w_q := w_q - V_q[:, 0:ncols] h_q   (h_q = h + q * hstride, on the device)
__global__ void sub_vh_kernel(int n, int Q, int ncols, const double *__restrict__ V, size_t vstride, int ldv,
                              const double *__restrict__ h, int hstride, double *__restrict__ w, size_t wstride) {
    const size_t total = (size_t)n * Q;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), q = (int)(e / n);
        const double *v = V + (size_t)q * vstride + i;
        const double *hq = h + (size_t)q * hstride;
        double acc = w[(size_t)q * wstride + i];
        for (int c = 0; c < ncols; ++c) acc = fma(-v[(size_t)c * ldv], hq[c], acc);
        w[(size_t)q * wstride + i] = acc;
    }
}

// y_q := a[q] * x_q
__global__ void scale_kernel(int n, int Q, const double *__restrict__ a, const double *__restrict__ x, size_t xstride,
                             double *__restrict__ y, size_t ystride) {
    const size_t total = (size_t)n * Q;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), q = (int)(e / n);
        y[(size_t)q * ystride + i] = a[q] * x[(size_t)q * xstride + i];
    }
}
// y[:, q] := fl32(x_q) for the active columns, 0 for the others
__global__ void to_f32_kernel(int n, int Q, const int *__restrict__ act, const double *__restrict__ x, size_t xstride,
                              float *__restrict__ y, int ldy) {
    const size_t total = (size_t)n * Q;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), q = (int)(e / n);
        y[(size_t)q * ldy + i] = act[q] ? (float)x[(size_t)q * xstride + i] : 0.f;
    }
}
__global__ void to_f64_kernel(int n, int Q, const float *__restrict__ x, int ldx, double *__restrict__ y, size_t ystride) {
    const size_t total = (size_t)n * Q;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), q = (int)(e / n);
        y[(size_t)q * ystride + i] = (double)x[(size_t)q * ldx + i];
    }
}
// x_q += Z_q[:, 0:k_q] y_q   (y_q = y + q * m, k on the device)
__global__ void add_zy_kernel(int n, int Q, const double *__restrict__ Z, size_t zstride, int ldz,
                              const double *__restrict__ y, const int *__restrict__ k, int m, double *__restrict__ X,
                              int ldx) {
    const size_t total = (size_t)n * Q;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), q = (int)(e / n);
        const double *z = Z + (size_t)q * zstride + i;
        double acc = 0.0;
        for (int c = 0; c < k[q]; ++c) acc = fma(z[(size_t)c * ldz], y[(size_t)q * m + c], acc);
        X[(size_t)q * ldx + i] += acc;
    }
}

static int g1(size_t total) { return (int)std::min<size_t>((total + 255) / 256, 152 * 8); }

static double b2d(unsigned long long b) {
    double d;
    memcpy(&d, &b, sizeof(d));
    return d;
}

static double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// FGMRES-IR on the right-hand side columns, kGmresChunk at a time.  On return
// X holds the refined solution and *eta_out the worst backward error.
// budget_ms > 0: stop (not converged) once that much host time has passed.
// Dinv (may be NULL): the FP32 factors' diagonal-block inverses for the
// preconditioner solves.
int gmres_ir(int n, int nrhs, const double *A, int lda, const double *B, int ldb, double *X, int ldx, const float *LU32,
             int ld32, const int *perm, double anorm, const double *bnorm, double tol, int max_outer, int restart,
             int *iters_out, int *inner_out, double *eta_out, cudaStream_t s, double budget_ms, const float *Dinv) {
    const auto t_start = std::chrono::steady_clock::now();
    const int m = std::max(1, restart);
    const int QM = std::min(nrhs, kGmresChunk);
    const size_t vs = (size_t)n * (m + 1), zs = (size_t)n * m;   // column strides of the V and Z families
    const int hs = m + 2;                                         // per-column stride of the device scalars
    double *V = nullptr, *Z = nullptr, *W = nullptr, *R = nullptr, *part = nullptr, *dv = nullptr, *dsc = nullptr;
    float *t32 = nullptr;
    int *dint = nullptr;   // [0, QM): active mask, [QM, 2 QM): k per column
    unsigned long long *nrm = nullptr;
    LU_CUDA_TRY(cudaMallocAsync(&V, sizeof(double) * vs * QM, s));
    LU_CUDA_TRY(cudaMallocAsync(&Z, sizeof(double) * zs * QM, s));
    LU_CUDA_TRY(cudaMallocAsync(&W, sizeof(double) * (size_t)n * QM, s));
    LU_CUDA_TRY(cudaMallocAsync(&R, sizeof(double) * (size_t)n * QM, s));
    LU_CUDA_TRY(cudaMallocAsync(&part, sizeof(double) * residual_workspace_doubles(n, QM), s));
    LU_CUDA_TRY(cudaMallocAsync(&dv, sizeof(double) * (size_t)hs * QM, s));
    LU_CUDA_TRY(cudaMallocAsync(&dsc, sizeof(double) * (size_t)m * QM, s));
    LU_CUDA_TRY(cudaMallocAsync(&t32, sizeof(float) * (size_t)n * QM, s));
    LU_CUDA_TRY(cudaMallocAsync(&dint, sizeof(int) * 2 * QM, s));
    LU_CUDA_TRY(cudaMallocAsync(&nrm, sizeof(unsigned long long) * 2 * QM, s));
    // every basis column starts finite: a column that stops early is only ever scaled by 0
    LU_CUDA_TRY(cudaMemsetAsync(V, 0, sizeof(double) * vs * QM, s));
    LU_CUDA_TRY(cudaMemsetAsync(Z, 0, sizeof(double) * zs * QM, s));
    int outer_total = 0, inner_total = 0;
    double worst = 0.0;
    bool out_of_time = false;
    // host state per column
    std::vector<double> H((size_t)QM * (m + 1) * m), cs((size_t)QM * m), sn((size_t)QM * m), g((size_t)QM * (m + 1));
    std::vector<double> h((size_t)QM * (m + 1)), beta(QM), eta(QM), hv((size_t)QM * hs), sc(QM), y((size_t)QM * m);
    std::vector<int> act(2 * QM), k(QM);
    std::vector<char> live(QM), inner(QM);
    std::vector<std::vector<double>> hist(QM);
    std::vector<unsigned long long> hn(2 * QM);
    for (int q0 = 0; q0 < nrhs && !out_of_time; q0 += QM) {
        const int Q = std::min(QM, nrhs - q0);
        double *Xc = X + (size_t)q0 * ldx;
        const double *Bc = B + (size_t)q0 * ldb;
        for (int q = 0; q < Q; ++q) { live[q] = 1; hist[q].clear(); eta[q] = INFINITY; }
        for (int outer = 0; outer <= max_outer; ++outer) {
            // r = b - A x and the backward error of every column
            LU_CUDA_TRY(launch_residual(n, Q, A, lda, Xc, ldx, Bc, ldb, R, n, part, nrm, s));
            LU_CUDA_TRY(launch_absmax(n, Q, Xc, ldx, nrm + Q, s));
            LU_CUDA_TRY(cudaMemcpyAsync(hn.data(), nrm, sizeof(unsigned long long) * 2 * Q, cudaMemcpyDeviceToHost, s));
            LU_CUDA_TRY(cudaStreamSynchronize(s));
            int nlive = 0;
            for (int q = 0; q < Q; ++q) {
                if (!live[q]) continue;
                const double den = anorm * b2d(hn[Q + q]) + bnorm[q0 + q];
                double e = den > 0 ? b2d(hn[q]) / den : 0.0;
                if (std::isnan(e)) e = INFINITY;
                eta[q] = e;
                hist[q].push_back(e);
                const size_t hsz = hist[q].size();
                if (e <= tol || outer == max_outer || (hsz >= 3 && !(hist[q][hsz - 1] <= 0.5 * hist[q][hsz - 3])))
                    live[q] = 0;   // converged, out of steps, or stalled
                else
                    ++nlive;
            }
            if (budget_ms > 0 && ms_since(t_start) > budget_ms) out_of_time = true;
            if (nlive == 0 || out_of_time) break;
            outer_total += nlive;
            // beta_q = ||r_q||_2, v_q0 = r_q / beta_q
            dots_kernel<<<dim3(1, Q), kDotThreads, 0, s>>>(n, 1, R, n, n, R, n, dv, hs);
            lu_count_launch();
            LU_CUDA_TRY(cudaMemcpyAsync(hv.data(), dv, sizeof(double) * hs * Q, cudaMemcpyDeviceToHost, s));
            LU_CUDA_TRY(cudaStreamSynchronize(s));
            for (int q = 0; q < Q; ++q) {
                beta[q] = std::sqrt(hv[(size_t)q * hs]);
                inner[q] = live[q] && beta[q] > 0.0 && std::isfinite(beta[q]);
                if (live[q] && !inner[q]) live[q] = 0;
                sc[q] = inner[q] ? 1.0 / beta[q] : 0.0;
                act[q] = inner[q];
                k[q] = 0;
                std::fill(g.begin() + (size_t)q * (m + 1), g.begin() + (size_t)(q + 1) * (m + 1), 0.0);
                g[(size_t)q * (m + 1)] = beta[q];
            }
            LU_CUDA_TRY(cudaMemcpyAsync(dsc, sc.data(), sizeof(double) * Q, cudaMemcpyHostToDevice, s));
            LU_CUDA_TRY(cudaMemcpyAsync(dint, act.data(), sizeof(int) * Q, cudaMemcpyHostToDevice, s));
            scale_kernel<<<g1((size_t)n * Q), 256, 0, s>>>(n, Q, dsc, R, n, V, vs);
            lu_count_launch();
            for (int j = 0; j < m; ++j) {
                int ninner = 0;
                for (int q = 0; q < Q; ++q) ninner += inner[q];
                if (ninner == 0) break;
                // z_qj = M^{-1} v_qj in FP32, kept in FP64; w_q = A z_qj in FP64
                to_f32_kernel<<<g1((size_t)n * Q), 256, 0, s>>>(n, Q, dint, V + (size_t)j * n, vs, t32, n);
                lu_count_launch();
                int rc = solve_f32_perm(n, Q, LU32, ld32, perm, t32, n, s, Dinv);
                if (rc != LU_OK) return rc;
                to_f64_kernel<<<g1((size_t)n * Q), 256, 0, s>>>(n, Q, t32, n, Z + (size_t)j * n, zs);
                lu_count_launch();
                LU_CUDA_TRY(launch_residual(n, Q, A, lda, Z + (size_t)j * n, (int)zs, nullptr, n, W, n, part, nrm, s));
                // classical Gram-Schmidt, twice
                std::fill(h.begin(), h.end(), 0.0);
                for (int pass = 0; pass < 2; ++pass) {
                    dots_kernel<<<dim3(j + 1, Q), kDotThreads, 0, s>>>(n, j + 1, V, vs, n, W, n, dv, hs);
                    lu_count_launch();
                    sub_vh_kernel<<<g1((size_t)n * Q), 256, 0, s>>>(n, Q, j + 1, V, vs, n, dv, hs, W, n);
                    lu_count_launch();
                    LU_CUDA_TRY(cudaMemcpyAsync(hv.data(), dv, sizeof(double) * hs * Q, cudaMemcpyDeviceToHost, s));
                    LU_CUDA_TRY(cudaStreamSynchronize(s));
                    for (int q = 0; q < Q; ++q)
                        for (int i = 0; i <= j; ++i) h[(size_t)q * (m + 1) + i] += hv[(size_t)q * hs + i];
                }
                dots_kernel<<<dim3(1, Q), kDotThreads, 0, s>>>(n, 1, W, n, n, W, n, dv, hs);
                lu_count_launch();
                LU_CUDA_TRY(cudaMemcpyAsync(hv.data(), dv, sizeof(double) * hs * Q, cudaMemcpyDeviceToHost, s));
                LU_CUDA_TRY(cudaStreamSynchronize(s));
                for (int q = 0; q < Q; ++q) {
                    const double hn2 = hv[(size_t)q * hs];
                    double *hq = h.data() + (size_t)q * (m + 1);
                    hq[j + 1] = std::sqrt(hn2);
                    sc[q] = (inner[q] && hq[j + 1] > 0.0) ? 1.0 / hq[j + 1] : 0.0;
                    if (!inner[q]) continue;
                    // apply the previous rotations, then a new one to zero h[j+1]
                    double *csq = cs.data() + (size_t)q * m, *snq = sn.data() + (size_t)q * m;
                    double *gq = g.data() + (size_t)q * (m + 1);
                    for (int i = 0; i < j; ++i) {
                        const double t = csq[i] * hq[i] + snq[i] * hq[i + 1];
                        hq[i + 1] = -snq[i] * hq[i] + csq[i] * hq[i + 1];
                        hq[i] = t;
                    }
                    const double den2 = std::hypot(hq[j], hq[j + 1]);
                    csq[j] = den2 > 0 ? hq[j] / den2 : 1.0;
                    snq[j] = den2 > 0 ? hq[j + 1] / den2 : 0.0;
                    hq[j] = den2;
                    hq[j + 1] = 0.0;
                    gq[j + 1] = -snq[j] * gq[j];
                    gq[j] = csq[j] * gq[j];
                    for (int i = 0; i <= j; ++i) H[((size_t)q * (m + 1) + i) * m + j] = hq[i];
                    k[q] = j + 1;
                    ++inner_total;
                    if (std::fabs(gq[j + 1]) <= 1e-10 * beta[q] || hn2 == 0.0) inner[q] = 0;
                }
                LU_CUDA_TRY(cudaMemcpyAsync(dsc, sc.data(), sizeof(double) * Q, cudaMemcpyHostToDevice, s));
                scale_kernel<<<g1((size_t)n * Q), 256, 0, s>>>(n, Q, dsc, W, n, V + (size_t)(j + 1) * n, vs);
                lu_count_launch();
                for (int q = 0; q < Q; ++q) act[q] = inner[q];
                LU_CUDA_TRY(cudaMemcpyAsync(dint, act.data(), sizeof(int) * Q, cudaMemcpyHostToDevice, s));
                if (budget_ms > 0 && ms_since(t_start) > budget_ms) break;   // keep the partial correction
            }
            // y_q = R_q^{-1} g_q (upper triangular back substitution), x_q += Z_q y_q
            for (int q = 0; q < Q; ++q) {
                const double *Hq = H.data() + (size_t)q * (m + 1) * m;
                const double *gq = g.data() + (size_t)q * (m + 1);
                double *yq = y.data() + (size_t)q * m;
                for (int i = k[q] - 1; i >= 0; --i) {
                    double t = gq[i];
                    for (int c = i + 1; c < k[q]; ++c) t -= Hq[(size_t)i * m + c] * yq[c];
                    yq[i] = Hq[(size_t)i * m + i] != 0.0 ? t / Hq[(size_t)i * m + i] : 0.0;
                }
                act[QM + q] = k[q];
            }
            LU_CUDA_TRY(cudaMemcpyAsync(dsc, y.data(), sizeof(double) * (size_t)m * Q, cudaMemcpyHostToDevice, s));
            LU_CUDA_TRY(cudaMemcpyAsync(dint + QM, act.data() + QM, sizeof(int) * Q, cudaMemcpyHostToDevice, s));
            add_zy_kernel<<<g1((size_t)n * Q), 256, 0, s>>>(n, Q, Z, zs, n, dsc, dint + QM, m, Xc, ldx);
            lu_count_launch();
            LU_CUDA_TRY(cudaStreamSynchronize(s));   // the host buffers are reused next cycle
        }
        for (int q = 0; q < Q; ++q) worst = std::max(worst, eta[q]);
    }
    if (out_of_time) worst = INFINITY;   // stopped by the budget: the caller measures the iterate again
    cudaFreeAsync(V, s);
    cudaFreeAsync(Z, s);
    cudaFreeAsync(W, s);
    cudaFreeAsync(R, s);
    cudaFreeAsync(part, s);
    cudaFreeAsync(dv, s);
    cudaFreeAsync(dsc, s);
    cudaFreeAsync(t32, s);
    cudaFreeAsync(dint, s);
    cudaFreeAsync(nrm, s);
    LU_CUDA_TRY(cudaGetLastError());
    *iters_out = outer_total;
    *inner_out = inner_total;
    *eta_out = worst;
    return LU_OK;
}

}  // namespace lu
