// Shared device/host helpers of liblu (CUDA path only).
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp8.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include "../../include/lu.h"

#define LU_CUDA_TRY(expr)                                                       \
    do {                                                                        \
        cudaError_t _e = (expr);                                                \
        if (_e != cudaSuccess) {                                                \
            lu_note_cuda_error(_e, #expr, __FILE__, __LINE__);                  \
            return LU_ERR_CUDA;                                                 \
        }                                                                       \
    } while (0)

void lu_note_cuda_error(cudaError_t e, const char *what, const char *file, int line);

// Library-wide device status word (LU_OK or LU_ERR_TIMEOUT), one per device.
int *lu_device_status_ptr();
// Counts kernel launches of this library (reported by lu_kernel_launches).
void lu_count_launch(int k = 1);
// Default bound for device-side waits, in globaltimer nanoseconds.
long long lu_spin_bound_ns(const lu_opts *o);
// SM count of the current device (looked up once per device; thread-safe).
cudaError_t lu_sm_count(int *sms);

__device__ __forceinline__ unsigned long long lu_globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int lu_ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void lu_st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int lu_ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded spin until *flag >= target: relaxed polls, then one acquire fence
// (an acquire on every poll would be needlessly expensive).  Returns false
// (and records LU_ERR_TIMEOUT in *status) when `bound_ns` of globaltimer time
// has passed.
__device__ __forceinline__ bool lu_wait_flag(const int *flag, int target, int *status, long long bound_ns) {
    if (lu_ld_relaxed(flag) < target) {
        const unsigned long long t0 = lu_globaltimer();
        unsigned int spins = 0;
        while (lu_ld_relaxed(flag) < target) {
            // back off: many pollers on one line would slow its writer down
            __nanosleep(spins < 8 ? 32 : 256);
            if (((++spins) & 7u) == 0u) {
                if ((long long)(lu_globaltimer() - t0) > bound_ns) {
                    atomicExch(status, (int)LU_ERR_TIMEOUT);
                    return false;
                }
            }
        }
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    return true;
}

// Per-CTA trace (lu_cta_trace): a kernel given a ring appends one record per
// CTA when it finishes.  tag = LU_TRACE_* kind << 24 | step.
struct CtaTrace {
    lu_cta_event *ring;   // device ring, nullptr when tracing is off
    int *count;           // device count of records made
    int cap;
    int tag;
};

__device__ __forceinline__ unsigned lu_smid() {
    unsigned r;
    asm volatile("mov.u32 %0, %smid;" : "=r"(r));
    return r;
}

// Called by one thread of the CTA at its end; t0 = %globaltimer at its start.
__device__ __forceinline__ void lu_trace_cta(const CtaTrace &tr, unsigned long long t0, int tiles) {
    if (!tr.ring) return;
    const int slot = atomicAdd(tr.count, 1);
    if (slot < tr.cap) {
        lu_cta_event e;
        e.kind = tr.tag >> 24;
        e.step = tr.tag & 0xffffff;
        e.cta = (int)blockIdx.x + (int)blockIdx.y * (int)gridDim.x;
        e.smid = (int)lu_smid();
        e.tiles = tiles;
        e.pad = 0;
        e.t0_ns = t0;
        e.t1_ns = lu_globaltimer();
        tr.ring[slot] = e;
    }
}

// Worker sharing between the panel branch and a persistent remainder update
// (section 4.1, malleable BLAS).  A persistent update holds one CTA per SM
// until its task queue is empty, so a panel cluster that reaches the GPU after
// it would wait for the whole update.  Before such a panel the panel branch
// raises *req; update CTAs on the SMs in mask (one cluster placement of the
// panel's size, found by lu_probe_cluster_sms) then stop taking tasks, which
// lets the cluster in; the panel clears *req when it starts, and a joining
// grid launched after the panel (mode 1) hands its SMs back to the queue.
//   mode 0: the launcher resets the task counter; 1: a joining grid of
//   join_ctas CTAs on a running update's counter; 2: the caller has reset it.
constexpr unsigned kShareMaskBits = 256;   // SM ids (%smid) a mask covers

struct SmShare {
    const int *req;
    const unsigned *mask;   // bit s % 32 of mask[s / 32]: SM s (kShareMaskBits bits)
    int mode;
    int join_ctas;
};

__device__ __forceinline__ bool lu_share_yield(const int *req, const unsigned *mask) {
    if (!req || !*reinterpret_cast<const volatile int *>(req)) return false;
    const unsigned s = lu_smid();
    return s < kShareMaskBits && ((mask[s >> 5] >> (s & 31u)) & 1u);
}

template <typename T> struct lu_abs_t;
template <> struct lu_abs_t<double> { __device__ static double f(double x) { return fabs(x); } };
template <> struct lu_abs_t<float>  { __device__ static float f(float x) { return fabsf(x); } };
template <typename T> __device__ __forceinline__ T lu_abs(T x) { return lu_abs_t<T>::f(x); }

// (|v|, row) maximum with the smallest row winning ties.  NaN magnitudes never
// win (comparisons with NaN are false), an invalid candidate has mag = -1.
template <typename T>
__device__ __forceinline__ bool lu_better(T mag_a, int idx_a, T mag_b, int idx_b) {
    return (mag_a > mag_b) || (mag_a == mag_b && idx_a < idx_b);
}

static inline int lu_ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Where and how the tensor-core update's operands are staged (the panel
// kernel stages L21, the interchange/solve kernel stages U12):
//   fmt 0: BF16; 1: BF16 hi | lo halves (hi at k, lo at kpad + k);
//   2: FP8 e4m3 scaled by a power of two per staged row or column, whose
//      inverse goes to scale[];
//   3: FP64 operands as kF64Slices BF16 digit slices (slice s at s * kpad + k,
//      see lu_f64_slices) with the power-of-two scale of each staged row or
//      column in dscale[].
// ptr == NULL: no staging.  lds and kpad count elements of the staged type.
// Early termination of a panel (section 4.2): the panel kernel reads *flag at
// the end of each inner panel and stops there when it equals epoch (force:
// stop at the first inner boundary whatever the flag); the width it factored
// goes to *w_out.  flag == nullptr and force == 0: the panel runs to its end.
struct EtArgs {
    const int *flag;
    int epoch;
    int force;
    int *w_out;
};

struct StageDesc {
    void *ptr;
    float *scale;
    int lds;
    int kpad;
    int fmt;
    double *dscale;
};

// Emulated FP64 products (Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012): an FP64
// row (or column) v with |v_k| < 2^e is written as
//   v_k = 2^e * sum_{s=0..6} x_{k,s} 2^{-8(s+1)} + r_k,  |r_k| <= 2^{e-57},
// with integer digits |x_{k,0}| <= 256, |x_{k,s}| <= 128 (s >= 1): the
// balanced base-256 digits of N_k = round(v_k 2^{56-e}), taken from the
// least significant end.  Digit s is stored pre-scaled, x_{k,s} 2^{-8(s+1)}:
// at most 8 significant bits, so exact in BF16, and the product of digits s
// and t lands at its natural scale 2^{-8(s+t+2)}.  The digits come from the
// bit fields of v with integer arithmetic (GB300's FP64 pipe is narrow).
constexpr int kF64Slices = 7;

// |x| as a bit pattern: non-negative doubles order like their patterns, so a
// row's largest magnitude is an integer maximum.
__device__ __forceinline__ unsigned long long lu_f64_abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// Exponent e of the scale 2^e of a row or column whose largest magnitude has
// pattern a: the least e with amax < 2^e (frexp's exponent), from the exponent
// field, or a subnormal's bit length; 0 for zero.  A row holding an infinity
// or a NaN gets e = 1025, so its scale 2^e is infinite and every result the
// row (or column) takes part in becomes infinite or NaN, as with FP64 FMAs,
// instead of losing the non-finite digits in the integer sums.
__device__ __forceinline__ int lu_f64_scale_exp_bits(unsigned long long a) {
    const int E = (int)(a >> 52);
    if (E == 0x7ff) return 1025;
    if (E) return E - 1022;
    const unsigned long long M = a & 0xfffffffffffffull;
    return M ? 64 - __clzll((long long)M) - 1074 : 0;
}

// The kF64Slices digits of x (|x| < 2^e) into out[s * stride], s = 0..6; a
// NaN or infinite x gives NaN digits.
template <typename BF>
__device__ __forceinline__ void lu_f64_slices(double x, int e, BF *out, size_t stride) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7ffu);
    if (E == 0x7ff) {
#pragma unroll
        for (int s = 0; s < kF64Slices; ++s) out[(size_t)s * stride] = __float2bfloat16_rn(__int_as_float(0x7fc00000));
        return;
    }
    unsigned long long M = b & 0xfffffffffffffull;
    if (E) M |= 1ull << 52;
    // |x| = M 2^{max(E,1) - 1075}, so N = round(|x| 2^{56-e}) = round(M 2^sh)
    const int sh = (E ? E : 1) - 1075 + 56 - e;
    long long N;
    if (M == 0 || sh <= -64) N = 0;
    else if (sh >= 0) N = sh < 64 ? (long long)(M << sh) : 0;              // M 2^sh < 2^56 as |x| < 2^e
    else N = (long long)((M + (1ull << (-sh - 1))) >> -sh);                // round half up
    if (b >> 63) N = -N;
    int d[kF64Slices];
#pragma unroll
    for (int s = kF64Slices - 1; s > 0; --s) {
        const int r = (int)((N + 128) & 255) - 128;   // balanced digit in [-128, 127]
        d[s] = r;
        N = (N - r) >> 8;                              // exact: N - r is a multiple of 256
    }
    d[0] = (int)N;                                     // |d0| <= 256
#pragma unroll
    for (int s = 0; s < kF64Slices; ++s)
        out[(size_t)s * stride] = __float2bfloat16_rn((float)d[s] * __int_as_float((127 - 8 * (s + 1)) << 23));
}

// Power-of-two scaling into the e4m3 range: the multiplier 2^e with the
// largest e such that amax * 2^e <= 448 (the largest finite e4m3 value), and
// its inverse; 1 for a zero or non-finite amax.  e is clamped so both stay
// normal FP32 numbers.
__device__ __forceinline__ float lu_fp8_scale(float amax, float *inv) {
    if (!(amax > 0.f) || !(amax <= 3.0e38f)) { *inv = 1.f; return 1.f; }
    int q = 0;
    const float mant = frexpf(amax, &q);            // amax = mant * 2^q, mant in [0.5, 1)
    int e = (mant <= 0.875f) ? 9 - q : 8 - q;       // 448 = 0.875 * 2^9
    e = e > 126 ? 126 : (e < -126 ? -126 : e);
    *inv = ldexpf(1.f, -e);
    return ldexpf(1.f, e);
}

__device__ __forceinline__ unsigned char lu_to_e4m3(float x) {
    return (unsigned char)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}

// Correctly rounded quotient x / d on a latency-critical chain, from a
// reciprocal computed beforehand off the chain: Markstein's correction
// (P. Markstein, "Computation of elementary functions on the IBM RISC
// System/6000 processor", IBM J. Res. Dev. 34(1), 1990): with rcp = RN(1/d)
// and q = RN(x * rcp) (within one ulp of x / d), the residual e = x - q d is
// exact in one fused multiply-add and RN(q + e rcp) = RN(x / d).  The
// theorem needs no overflow or underflow in these steps: lu_div_safe tells
// whether |d| and |x| (or x = 0) lie well inside the exponent range; callers
// redo the rare unsafe cases with the IEEE division.
template <typename T> struct lu_div_range;
template <> struct lu_div_range<float> {
    static constexpr unsigned lo = (127u - 60u) << 23, hi = (127u + 60u) << 23;   // 2^-60 .. 2^60
    __device__ static bool in(float v) {
        const unsigned b = __float_as_uint(v) & 0x7fffffffu;
        return b >= lo && b < hi;
    }
};
template <> struct lu_div_range<double> {
    static constexpr unsigned long long lo = (1023ull - 500ull) << 52, hi = (1023ull + 500ull) << 52;   // 2^-500 .. 2^500
    __device__ static bool in(double v) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
        return b >= lo && b < hi;
    }
};

template <typename T>
__device__ __forceinline__ bool lu_div_safe(T x, bool ok_d) {
    return ok_d && (x == T(0) || lu_div_range<T>::in(x));
}

template <typename T>
__device__ __forceinline__ T lu_div_fast(T x, T d, T rcp) {
    const T q = x * rcp;
    return fma(fma(-q, d, x), rcp, q);
}
