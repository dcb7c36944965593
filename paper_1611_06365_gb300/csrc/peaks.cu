// Throughput probes of the arithmetic units the FP64 and FP32 paths run on,
// used as measured roofline denominators (lu_peak_probe in lu.h).
//
//   kind 0  DFMA: FP64 fused multiply-adds on the CUDA cores (the FP64 update,
//           the FP64 panel and the batched FP64 kernel use these)
//   kind 1  FFMA: FP32 fused multiply-adds (the FP32 SIMT kernels)
//   kind 2  DMMA: mma.sync m8n8k4 with FP64 operands (the legacy FP64 tensor
//           path; tcgen05 has no FP64 kind)
//
// The DFMA probe runs the compute loop of the tiled update (a 4 x 4 outer
// product per thread per step of K, operands from shared memory, 16
// independent accumulators), the FFMA probe 8 independent register chains per
// thread, and every DMMA warp 4 chains; the grid holds kCtasPerSm CTAs of 256
// threads per SM.  The accumulators grow linearly from
// small positive products, so nothing overflows or goes subnormal, and a
// data-dependent store keeps the compiler from removing the work.
#include "common.cuh"

namespace lu {

constexpr int kProbeThreads = 256;
constexpr int kProbeCtasPerSm = 4;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe(long long iters, T m, T c, T *sink) {
    // the inner loop of the tiled update (gemm_simt.cu) without its global
    // traffic: a 64 x 64 tile, 4 x 4 outputs per thread, operands read from
    // shared memory at every step of K
    constexpr int TM = 64, TN = 64, TX = TM / 4, TY = TN / 4;
    __shared__ T As[16][TM];
    __shared__ T Bs[16][TN + 1];
    for (int e = threadIdx.x; e < 16 * TM; e += kProbeThreads) As[e / TM][e % TM] = m * T(1 + (e & 7));
    for (int e = threadIdx.x; e < 16 * (TN + 1); e += kProbeThreads) Bs[e / (TN + 1)][e % (TN + 1)] = c * T(1 + (e & 3));
    __syncthreads();
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + TX * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + TY * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();   // as between the update's K chunks (and the operands are read again)
    }
    T s = T(0);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) s += acc[i][j];
    if (s == T(-1)) sink[blockIdx.x] = s;   // never true: every term is positive
}

// Independent FMA chains (8 per thread) on operands held in registers: the
// pattern that reaches the FP32 pipe's rate (the tile loop above is bound by
// its shared-memory operand loads in FP32, not in FP64).
template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_chains(long long iters, T m, T c, T *sink) {
    T a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = T(threadIdx.x + i) * T(1e-3);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fma(a[i], m, c);
    }
    T s = T(0);
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == T(-1)) sink[blockIdx.x] = s;   // never true: the chains stay positive
}

__global__ void __launch_bounds__(kProbeThreads) dmma_probe(long long iters, double m, double *sink) {
    double d[4][2];
    const double a = m, b = 1.0 - 1e-3 * (threadIdx.x & 7);
#pragma unroll
    for (int i = 0; i < 4; ++i) { d[i][0] = 1e-3 * i; d[i][1] = 2e-3 * i; }
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            // D = A B + C on an 8x8x4 tile per warp; the accumulator feeds back
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(d[i][0]), "+d"(d[i][1])
                         : "d"(a), "d"(b));
        }
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) s += d[i][0] + d[i][1];
    if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace lu

extern "C" int lu_peak_probe(int kind, long long iters, double *tflops, double *ms_out, void *stream) {
    if (kind < 0 || kind > 2) return -1;
    if (iters <= 0) return -2;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    LU_CUDA_TRY(cudaGetDevice(&dev));
    LU_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * lu::kProbeCtasPerSm;
    void *sink = nullptr;
    LU_CUDA_TRY(cudaMallocAsync(&sink, (size_t)grid * sizeof(double), s));
    cudaEvent_t e0, e1;
    LU_CUDA_TRY(cudaEventCreate(&e0));
    LU_CUDA_TRY(cudaEventCreate(&e1));
    LU_CUDA_TRY(cudaEventRecord(e0, s));
    double flops = 0.0;
    const double threads = (double)grid * lu::kProbeThreads;
    if (kind == 0) {
        lu::fma_probe<double><<<grid, lu::kProbeThreads, 0, s>>>(iters, 0.999, 1e-3, static_cast<double *>(sink));
        flops = threads * (double)iters * 16 * 16 * 2.0;
    } else if (kind == 1) {
        lu::fma_chains<float><<<grid, lu::kProbeThreads, 0, s>>>(iters, 0.999f, 1e-3f, static_cast<float *>(sink));
        flops = threads * (double)iters * 8 * 2.0;
    } else {
        lu::dmma_probe<<<grid, lu::kProbeThreads, 0, s>>>(iters, 0.5, static_cast<double *>(sink));
        flops = threads / 32.0 * (double)iters * 4.0 * (2.0 * 8 * 8 * 4);
    }
    lu_count_launch();
    LU_CUDA_TRY(cudaGetLastError());
    LU_CUDA_TRY(cudaEventRecord(e1, s));
    LU_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    LU_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    LU_CUDA_TRY(cudaFreeAsync(sink, s));
    LU_CUDA_TRY(cudaStreamSynchronize(s));
    if (tflops) *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    if (ms_out) *ms_out = ms;
    return LU_OK;
}
