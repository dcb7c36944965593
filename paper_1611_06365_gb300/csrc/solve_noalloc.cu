// lu_solve_noalloc: the triangular solves of lu_solve with no memory
// allocation at all.
//
// Who needs it: callers that must not allocate device memory during a solve.
// Typical cases are an application whose framework has already reserved the
// device memory for its own pool, so that any extra cudaMalloc fails with an
// out-of-memory error, and a latency-critical loop where an allocation may
// stall waiting for the device.  lu_solve allocates its workspace
// (permutation vector, a copy of B, the wait flags of the blocked substitution)
// stream-ordered on every call; this entry point takes the same workspace from
// a fixed array in device memory instead.
//
// The array is a file-scope __device__ variable of kNoAllocScratchBytes bytes:
// every GPU that loads liblu holds it until the process exits.  In host code
// the variable's name is only a host-side stand-in, so its device address is
// looked up with cudaGetSymbolAddress, once per device, with that device
// current, on the first call made on that device; that first call should
// therefore happen before any stream capture.  All calls share the one array
// and it keeps the last call's contents: each call clears the parts that must
// start at zero (the wait flags and the status word), and two calls whose
// work overlaps on the GPU (different streams, or different host threads)
// race on it -- serialize them.
#include "common.cuh"
#include <algorithm>
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)4 << 20;   // 4 MiB per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {nullptr};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Bytes of scratch a request needs: status word, flags of the blocked
// substitution, permutation vector, permuted copy of B.
size_t scratch_bytes(int n, int nrhs, size_t elem) {
    return align256(sizeof(int)) + align256(lu::trsv_workspace_ints(n, nrhs) * sizeof(int)) + align256((size_t)n * sizeof(int)) +
           align256((size_t)n * nrhs * elem);
}

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(unsigned char **out) {
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    if (d < 0 || d >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[d]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[d] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[d];
    return cudaSuccess;
}

template <typename T>
int solve_noalloc(int n, int nrhs, const T *LU, int lda, const int *ipiv, T *B, int ldb, int *d_status, cudaStream_t s) {
    unsigned char *base = nullptr;
    LU_CUDA_TRY(scratch_address(&base));
    int *status = reinterpret_cast<int *>(base);
    size_t off = align256(sizeof(int));
    int *tws = reinterpret_cast<int *>(base + off);
    off += align256(lu::trsv_workspace_ints(n, nrhs) * sizeof(int));
    int *perm = reinterpret_cast<int *>(base + off);
    off += align256((size_t)n * sizeof(int));
    T *X = reinterpret_cast<T *>(base + off);
    int dev = 0, sms = 0;
    LU_CUDA_TRY(cudaGetDevice(&dev));
    LU_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LU_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    LU_CUDA_TRY(lu::launch_ipiv_to_perm(ipiv, n, perm, s));
    LU_CUDA_TRY((lu::launch_gather_rows<T, T>(n, nrhs, perm, B, ldb, X, n, s)));
    // launch_trsv_pair clears its flags and tickets before the two sweeps
    LU_CUDA_TRY(lu::launch_trsv_pair<T>(LU, lda, n, nrhs, X, n, tws, status, lu_spin_bound_ns(nullptr), sms, s));
    LU_CUDA_TRY(cudaMemcpy2DAsync(B, sizeof(T) * ldb, X, sizeof(T) * n, sizeof(T) * n, nrhs, cudaMemcpyDeviceToDevice, s));
    if (d_status) LU_CUDA_TRY(cudaMemcpyAsync(d_status, status, sizeof(int), cudaMemcpyDeviceToDevice, s));
    return LU_OK;
}

}  // namespace

extern "C" size_t lu_solve_noalloc_capacity(void) { return kNoAllocScratchBytes; }

extern "C" int lu_solve_noalloc(lu_dtype dt, int n, int nrhs, const void *dLU, int lda, const int *d_ipiv, void *dB, int ldb,
                                int *d_status, void *stream) {
    if (dt != LU_F64 && dt != LU_F32) return -1;
    if (n < 0) return -2;
    if (nrhs < 0) return -3;
    if (n > 0 && !dLU) return -4;
    if (lda < std::max(1, n)) return -5;
    if (n > 0 && !d_ipiv) return -6;
    if (n > 0 && nrhs > 0 && !dB) return -7;
    if (ldb < std::max(1, n)) return -8;
    const size_t elem = dt == LU_F64 ? sizeof(double) : sizeof(float);
    if (scratch_bytes(n, nrhs, elem) > kNoAllocScratchBytes) return LU_ERR_SCRATCH;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0 || nrhs == 0) {
        if (d_status) LU_CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int), s));
        return LU_OK;
    }
    if (dt == LU_F64)
        return solve_noalloc<double>(n, nrhs, static_cast<const double *>(dLU), lda, d_ipiv, static_cast<double *>(dB), ldb,
                                     d_status, s);
    return solve_noalloc<float>(n, nrhs, static_cast<const float *>(dLU), lda, d_ipiv, static_cast<float *>(dB), ldb,
                                d_status, s);
}
