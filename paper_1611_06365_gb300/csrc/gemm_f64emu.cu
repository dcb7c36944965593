// Emulated FP64 trailing update RL3 / PF2 / RU2 (section 3.1, Figure 1 right;
// section 3.2, Figure 3) on the 5th-generation tensor cores:
//   C := C - A B,  C FP64 (m x n, column-major), A = L21 (m x K), B = U12 (K x n),
// with A and B given as BF16 digit slices (lu_f64_slices in common.cuh: seven
// 8-bit digits per entry below a power-of-two scale per row of A and per
// column of B).  The product is the error-free splitting of Ozaki, Ogita,
// Oishi and Rump (Numer. Algorithms 59, 2012): A B = sum over digit pairs
// (s, t) of A_s B_t, every A_s B_t an exact integer multiple of
// 2^{-8(s+t+2)}.  The pairs with s + t <= 6 are kept (28 products):
//   * pairs with s + t = 0 .. 4 are summed per diagonal d = s + t in their
//     own FP32 TMEM accumulator; with K <= 64 every partial sum is an
//     integer multiple of 2^{-8(d+2)} of magnitude below 2^24 of those units,
//     so the tensor core's FP32 accumulation is exact;
//   * pairs with s + t = 5 and 6 share a sixth accumulator, rounded in FP32.
// In units of the two scales' product 2^{e_i + e_j}, with K = 64: a dropped
// pair (s + t >= 7) is at most 2^-58 per k, all of them together below
// 2^-49.4, and the sixth accumulator's rounding below 2^-50.7 (worst cases;
// a K-term DFMA chain may round by K^2 2^-53 = 2^-41 of the same units).
// The epilogue adds the six accumulators exactly in a 64-bit integer (units of
// 2^-56 of the scales' product; the shared accumulator rounded to that unit),
// converts it to FP64 (one rounding), multiplies it by the column's
// power-of-two scale by adding to its exponent field, and subtracts it from C
// with one fused multiply-add by the row's scale: two roundings per element,
// against K for a DFMA chain, and two FP64-pipe operations per element (a
// column scale outside the exponent-add range takes an FP64 multiply instead).
// The scales are per row and column,
// so a row whose entries differ widely in magnitude keeps the absolute, not
// the relative, accuracy of its largest entry (the normwise property of the
// splitting).
//
// Persistent, warp-specialized kernel, one CTA per SM.  A task is a 128-row
// block times up to kEmMaxSub sub-tiles of 32 columns, taken from a global
// atomic queue; the task's A slices (7 x 16 KB) stay in shared memory while
// its sub-tiles stream through:
//   warp 0   TMA producer: A slices once per task, B slices (7 x 4 KB) per
//            sub-tile into a two-stage ring;
//   warp 1   MMA issuer (one thread): 28 products x 4 K-steps of
//            tcgen05.mma kind::f16 (M = 128, N = 32, K = 16) into one of two
//            sets of six TMEM accumulators (2 x 6 x 32 columns);
//   warps 2-17 epilogue: load the sub-tile's C while the MMAs run, read the
//            accumulators (tcgen05.ld), combine them in integer arithmetic,
//            store C (four warps per TMEM lane quarter, 8 columns each: the
//            epilogue is latency-bound, so more warps at fewer registers each).
// Every wait is bounded; on expiry the kernel records LU_ERR_TIMEOUT, gives
// its copies in flight one bounded wait, frees its TMEM and returns.
#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"
#include <cuda_bf16.h>

namespace lu {

constexpr int kEmBM = 128;
constexpr int kEmBN = 32;
constexpr int kEmK = 64;                       // K per slice: one 128-byte swizzle span of BF16
constexpr int kEmAcc = 6;
constexpr int kEmMaxSub = 8;
constexpr int kEmEpiWarps = 16;               // epilogue warps: four per TMEM lane quarter
constexpr int kEmEpiCols = kEmBN * 4 / kEmEpiWarps;   // sub-tile columns per epilogue warp (8)
constexpr int kEmThreads = 64 + 32 * kEmEpiWarps;     // TMA, MMA, epilogue
constexpr int kEmSliceA = kEmBM * kEmK * 2;    // 16 KB
constexpr int kEmSliceB = kEmBN * kEmK * 2;    // 4 KB
constexpr int kEmStageB = kF64Slices * kEmSliceB;
constexpr int kEmStagesB = 2;
constexpr uint32_t kEmTmemCols = 512;          // 2 x 6 x 32 used
constexpr size_t kEmSmem = 1024 + (size_t)kF64Slices * kEmSliceA + (size_t)kEmStagesB * kEmStageB + 512;
constexpr int kEmLast = 1 << 16;               // sub-tile flag: last of its task

__global__ void __launch_bounds__(kEmThreads, 1)
gemm_update_f64emu(int m, int n, const __grid_constant__ CUtensorMap mapA, int a_row0,
                   const __grid_constant__ CUtensorMap mapB, int b_col0, double *__restrict__ C, int ldc,
                   const double *__restrict__ scaleA, const double *__restrict__ scaleB, int nsub, int lshift,
                   int *__restrict__ tile_ctr, int *__restrict__ status, long long bound_ns, CtaTrace tr,
                   const int *__restrict__ yreq, const unsigned *__restrict__ ymask) {
    const unsigned long long t_start = tr.ring ? lu_globaltimer() : 0ull;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (base - raw);
    const uint32_t sA = base;                                              // 7 slices x 16 KB
    const uint32_t sB = base + (uint32_t)kF64Slices * kEmSliceA;           // 2 stages x 7 slices x 4 KB
    uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + (size_t)kF64Slices * kEmSliceA + (size_t)kEmStagesB * kEmStageB);
    // bars: a_full, a_empty, b_full[2], b_empty[2], acc_full[2], acc_empty[2], tile_full[2]
    const uint32_t a_full = smem_u32(bars), a_empty = a_full + 8u;
    const uint32_t b_full0 = a_empty + 8u, b_empty0 = b_full0 + 8u * kEmStagesB;
    const uint32_t accf0 = b_empty0 + 8u * kEmStagesB, acce0 = accf0 + 16u, tilef0 = acce0 + 16u;
    int *ints = reinterpret_cast<int *>(bars + 4 + 4 * kEmStagesB);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(ints);
    volatile int *abort_flag = ints + 1;
    volatile int *stage_task = ints + 2;                  // [kEmStagesB]
    volatile int *stage_sub = ints + 2 + kEmStagesB;      // [kEmStagesB]
    volatile int *acc_task = ints + 2 + 2 * kEmStagesB;   // [2]
    volatile int *acc_sub = ints + 4 + 2 * kEmStagesB;    // [2]
    volatile int *issued = ints + 6 + 2 * kEmStagesB;     // [1 + kEmStagesB]: parity of a load in flight + 1, 0 none
    volatile int *ntasks_done = ints + 7 + 3 * kEmStagesB; // tasks this CTA took

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = (m + kEmBM - 1) / kEmBM;
    const int cols_task = kEmBN * nsub;
    const int ntasks = mt * ((n + cols_task - 1) / cols_task);

    // a CTA that starts after the queue ran dry (the tail of a joining grid), or on
    // an SM the panel branch asked back, leaves before claiming TMEM
    __shared__ int leave;
    if (tid == 0) leave = *reinterpret_cast<volatile int *>(tile_ctr) >= ntasks || lu_share_yield(yreq, ymask);
    __syncthreads();
    if (leave) {
        if (tid == 0) lu_trace_cta(tr, t_start, 0);
        return;
    }

    if (tid == 0) {
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        for (int i = 0; i < kEmStagesB; ++i) { mbar_init(b_full0 + 8u * i, 1); mbar_init(b_empty0 + 8u * i, 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(accf0 + 8u * i, 1); mbar_init(acce0 + 8u * i, 32 * kEmEpiWarps); mbar_init(tilef0 + 8u * i, 1); }
        *abort_flag = 0;
        for (int i = 0; i <= kEmStagesB; ++i) issued[i] = 0;
        *ntasks_done = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kEmTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int sb = 0;
            uint32_t bph = 0, aph = 0;
            for (;;) {
                // worker sharing: on the panel's SMs, stop at a task boundary when asked
                int t = lu_share_yield(yreq, ymask) ? -1 : atomicAdd(tile_ctr, 1);
                if (t >= ntasks || *abort_flag) t = -1;
                int nj = 0, tm = 0, tn = 0;
                while (t >= 0) {
                    tm = (t % mt) * kEmBM;
                    tn = (t / mt) * cols_task;
                    nj = min(nsub, (n - tn + kEmBN - 1) / kEmBN);
                    // lower-triangle updates: only the sub-tiles reaching the kept triangle
                    if (lshift >= 0) nj = min(nj, tm + kEmBM - 1 - lshift - tn < 0 ? 0 : (tm + kEmBM - 1 - lshift - tn) / kEmBN + 1);
                    if (nj > 0) break;
                    t = atomicAdd(tile_ctr, 1);
                    if (t >= ntasks || *abort_flag) t = -1;
                }
                if (t >= 0) {
                    *ntasks_done = *ntasks_done + 1;
                    // the previous task's MMAs must be done with the A slices
                    if (!mbar_wait_bounded(a_empty, aph ^ 1u, bound_ns)) { *abort_flag = 1; t = -1; }
                    else {
                        mbar_expect_tx(a_full, (uint32_t)kF64Slices * kEmSliceA);
                        issued[0] = (int)aph + 1;
#pragma unroll
                        for (int s = 0; s < kF64Slices; ++s)
                            tma_load_2d(sA + (uint32_t)s * kEmSliceA, &mapA, s * kEmK, a_row0 + tm, a_full);
                        aph ^= 1u;
                        for (int j = 0; j < nj; ++j) {
                            if (!mbar_wait_bounded(b_empty0 + 8u * sb, bph ^ 1u, bound_ns)) { *abort_flag = 1; break; }
                            const uint32_t fb = b_full0 + 8u * sb, st = sB + (uint32_t)sb * kEmStageB;
                            stage_task[sb] = t;
                            stage_sub[sb] = j | (j == nj - 1 ? kEmLast : 0);
                            mbar_expect_tx(fb, (uint32_t)kEmStageB);
                            issued[1 + sb] = (int)bph + 1;
#pragma unroll
                            for (int s = 0; s < kF64Slices; ++s)
                                tma_load_2d(st + (uint32_t)s * kEmSliceB, &mapB, s * kEmK, b_col0 + tn + j * kEmBN, fb);
                            if (++sb == kEmStagesB) { sb = 0; bph ^= 1u; }
                        }
                        if (*abort_flag) t = -1;
                    }
                }
                if (t < 0) {
                    // end of the queue: a stage with task -1 tells the MMA warp
                    if (mbar_wait_bounded(b_empty0 + 8u * sb, bph ^ 1u, bound_ns)) {
                        stage_task[sb] = -1;
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b_full0 + 8u * sb) : "memory");
                    } else {
                        *abort_flag = 1;
                    }
                    break;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = umma_idesc_bf16(kEmBM, kEmBN);
            int sb = 0;
            uint32_t bph = 0, aph = 0;
            for (int it = 0;; ++it) {
                const int a = it & 1;
                const uint32_t acc_ph = (uint32_t)((it >> 1) & 1);
                bool stop = false;
                int t = -1, sub = 0;
                if (!mbar_wait_bounded(b_full0 + 8u * sb, bph, bound_ns)) { *abort_flag = 1; stop = true; }
                else { t = stage_task[sb]; sub = stage_sub[sb]; }
                // the accumulator must be free before its task index is replaced, the end
                // marker included: tile_full may run at most one phase ahead of the epilogue
                if (!stop && !mbar_wait_bounded(acce0 + 8u * a, acc_ph ^ 1u, bound_ns)) { *abort_flag = 1; stop = true; }
                if (!stop && t >= 0 && (sub & (kEmLast - 1)) == 0) {
                    if (!mbar_wait_bounded(a_full, aph, bound_ns)) { *abort_flag = 1; stop = true; }
                    aph ^= 1u;
                }
                if (stop || t < 0 || *abort_flag) {
                    acc_task[a] = -1;
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tilef0 + 8u * a) : "memory");
                    break;
                }
                acc_task[a] = t;
                acc_sub[a] = sub;
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tilef0 + 8u * a) : "memory");
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t accb = tmem + (uint32_t)(a * kEmAcc * kEmBN);
                // descriptors of the slices' first K-step; later ones add their byte offset / 16
                // to the start-address field (every operand lies below 256 KB of shared memory)
                const uint64_t dA0 = umma_desc_sw128(sA), dB0 = umma_desc_sw128(sB + (uint32_t)sb * kEmStageB);
                bool started[kEmAcc] = {false, false, false, false, false, false};
#pragma unroll
                for (int s = 0; s < kF64Slices; ++s) {
#pragma unroll
                    for (int u = 0; u < kF64Slices - s; ++u) {
                        const int g = s + u < kEmAcc - 1 ? s + u : kEmAcc - 1;
#pragma unroll
                        for (int kk = 0; kk < kEmK / 16; ++kk) {
                            umma_bf16(accb + (uint32_t)(g * kEmBN), dA0 + (uint64_t)((s * kEmSliceA + kk * 32) >> 4),
                                      dB0 + (uint64_t)((u * kEmSliceB + kk * 32) >> 4), idesc, started[g] ? 1u : 0u);
                            started[g] = true;
                        }
                    }
                }
                umma_commit(b_empty0 + 8u * sb);                // B stage free once these MMAs are done
                if (sub & kEmLast) umma_commit(a_empty);        // A slices free after the task's last sub-tile
                umma_commit(accf0 + 8u * a);                    // accumulators ready
                if (++sb == kEmStagesB) { sb = 0; bph ^= 1u; }
            }
        }
    } else {
        // epilogue: warps 2..17; warp w reads TMEM lane quarter w % 4 (thread = tile row) and
        // handles kEmEpiCols of the sub-tile's 32 columns (h = (w - 2) / 4: the column group)
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int r = q * 32 + lane;
        for (int it = 0;; ++it) {
            const int a = it & 1;
            const uint32_t acc_ph = (uint32_t)((it >> 1) & 1);
            if (!mbar_wait_bounded(tilef0 + 8u * a, acc_ph, bound_ns)) { *abort_flag = 1; break; }
            const int t = acc_task[a];
            if (t < 0) break;
            const int j = acc_sub[a] & (kEmLast - 1);
            const int row = (t % mt) * kEmBM + r;
            const int col0 = (t / mt) * cols_task + j * kEmBN + h * kEmEpiCols;
            const bool rok = row < m;
            // this sub-tile's C, loaded while its products are formed
            double cv[kEmEpiCols];
            double *crow = C + (size_t)(rok ? row : 0);
#pragma unroll
            for (int c = 0; c < kEmEpiCols; ++c) cv[c] = (rok && col0 + c < n) ? crow[(size_t)(col0 + c) * ldc] : 0.0;
            // the row's scale times 2^-56, the unit of the integer sum below
            const double sa56 = rok ? scaleA[a_row0 + row] * 0x1p-56 : 0.0;
            if (!mbar_wait_bounded(accf0 + 8u * a, acc_ph, bound_ns) || *abort_flag) { *abort_flag = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t accb = tmem + (uint32_t)(a * kEmAcc * kEmBN + h * kEmEpiCols) + ((uint32_t)(q * 32) << 16);
            // The six accumulators combined exactly in a 64-bit integer in units of 2^-56
            // (on the integer and FP32 pipes; GB300's FP64 pipe is narrow): diagonal g <= 4
            // holds an integer multiple of 2^{-8(g+2)} below 2^24 of those units, so
            // acc_g * 2^{8(g+2)} converts exactly and scales by 2^{40-8g}; the shared sixth
            // accumulator is rounded to the unit (at most 2^-57 of the scales' product; its
            // magnitude stays below 2^24 units, so a 32-bit conversion holds it).
            // |sum| < 2^63; one conversion to FP64 and one FMA then give C - A B.
            long long vi[kEmEpiCols];
#pragma unroll
            for (int c = 0; c < kEmEpiCols; ++c) vi[c] = 0;
#pragma unroll
            for (int g = 0; g < kEmAcc; ++g) {
                float f[kEmEpiCols];
                tmem_ld8(accb + (uint32_t)(g * kEmBN), f);
                if (g < kEmAcc - 1) {
                    const float up = __int_as_float((127 + 8 * (g + 2)) << 23);   // 2^{8(g+2)}
                    const long long mul = 1LL << (40 - 8 * g);
#pragma unroll
                    for (int c = 0; c < kEmEpiCols; ++c) vi[c] += (long long)__float2int_rz(f[c] * up) * mul;
                } else {
#pragma unroll
                    for (int c = 0; c < kEmEpiCols; ++c) vi[c] += (long long)__float2int_rn(f[c] * 0x1p56f);
                }
            }
            // Column scales 2^eb: a nonzero converted sum has a biased exponent in [1023, 1085],
            // so adding eb to it stays a normal number for biased eb in [1, 1984].  The warp's
            // columns are the same for every lane, so the choice is made once for all of them
            // (a branch per column would be if-converted and issue both paths).
            bool fast = true;
#pragma unroll
            for (int c = 0; c < kEmEpiCols; ++c) {
                const int eb = (int)((__double_as_longlong(__ldg(&scaleB[b_col0 + min(col0 + c, n - 1)])) >> 52) & 0x7ff);
                fast = fast && eb >= 1 && eb <= 1984;
            }
            if (fast) {
#pragma unroll
                for (int c = 0; c < kEmEpiCols; ++c) {
                    const int eb = (int)((__double_as_longlong(__ldg(&scaleB[b_col0 + min(col0 + c, n - 1)])) >> 52) & 0x7ff);
                    const long long db = __double_as_longlong(__ll2double_rn(vi[c]));
                    cv[c] = fma(-__longlong_as_double(db == 0 ? 0 : db + (long long)(eb - 1023) * (1LL << 52)), sa56, cv[c]);
                }
            } else {
                // the scales' product first: the converted sum times a column scale above 2^961
                // may overflow
#pragma unroll
                for (int c = 0; c < kEmEpiCols; ++c)
                    cv[c] = fma(-(sa56 * __ldg(&scaleB[b_col0 + min(col0 + c, n - 1)])), __ll2double_rn(vi[c]), cv[c]);
            }
            // accumulators read: the MMAs of the sub-tile after next may start
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce0 + 8u * a) : "memory");
#pragma unroll
            for (int c = 0; c < kEmEpiCols; ++c)
                if (rok && col0 + c < n && (lshift < 0 || row >= col0 + c + lshift)) crow[(size_t)(col0 + c) * ldc] = cv[c];
        }
    }
    __syncthreads();
    if (tid == 0 && *abort_flag) {
        atomicExch(status, (int)LU_ERR_TIMEOUT);
        // give copies in flight one bounded chance to land before shared memory is released
        if (issued[0]) mbar_wait_bounded(a_full, (uint32_t)(issued[0] - 1), bound_ns / 4);
        for (int i = 0; i < kEmStagesB; ++i)
            if (issued[1 + i]) mbar_wait_bounded(b_full0 + 8u * i, (uint32_t)(issued[1 + i] - 1), bound_ns / 4);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kEmTmemCols) : "memory");
    }
    if (tid == 0) lu_trace_cta(tr, t_start, *ntasks_done);
}

// ---- operand staging (standalone; inside the factorization the panel kernel
// stages L21 and the interchange/solve kernel stages U12) ---------------------

// L (rows x k, FP64 column-major, ld) -> digit slices stage[i * lds + s * kpad + kk]
// (zero for kk in [k, kpad)) and scale[i] = 2^e_i.  One warp per row.
__global__ void stage_rows_f64emu(int rows, int k, int kpad, const double *__restrict__ L, int ld,
                                  __nv_bfloat16 *__restrict__ stage, int lds, double *__restrict__ scale) {
    const int lane = threadIdx.x & 31;
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < rows; i += gridDim.x * (blockDim.x >> 5)) {
        unsigned long long amax = 0;
        for (int kk = lane; kk < k; kk += 32) amax = max(amax, lu_f64_abs_bits(L[(size_t)i + (size_t)kk * ld]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        const int e = lu_f64_scale_exp_bits(amax);
        if (lane == 0) scale[i] = ldexp(1.0, e);
        for (int kk = lane; kk < kpad; kk += 32)
            lu_f64_slices(kk < k ? L[(size_t)i + (size_t)kk * ld] : 0.0, e, stage + (size_t)i * lds + kk, (size_t)kpad);
    }
}

// B (k x cols, FP64 column-major, ld) -> digit slices stage[j * lds + s * kpad + kk], scale[j].
__global__ void stage_cols_f64emu(int k, int kpad, int cols, const double *__restrict__ B, int ld,
                                  __nv_bfloat16 *__restrict__ stage, int lds, double *__restrict__ scale) {
    const int lane = threadIdx.x & 31;
    for (int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < cols; j += gridDim.x * (blockDim.x >> 5)) {
        unsigned long long amax = 0;
        for (int kk = lane; kk < k; kk += 32) amax = max(amax, lu_f64_abs_bits(B[(size_t)kk + (size_t)j * ld]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        const int e = lu_f64_scale_exp_bits(amax);
        if (lane == 0) scale[j] = ldexp(1.0, e);
        for (int kk = lane; kk < kpad; kk += 32)
            lu_f64_slices(kk < k ? B[(size_t)kk + (size_t)j * ld] : 0.0, e, stage + (size_t)j * lds + kk, (size_t)kpad);
    }
}

// ---- host side -----------------------------------------------------------------

int f64emu_kpad() { return kEmK; }
int f64emu_box_rows() { return kEmBM; }
int f64emu_box_cols() { return kEmBN; }

// C[m x n] -= A[a_row0 + (0..m), 0..K) B[0..K, b_col0 + (0..n)] with A and B as
// digit slices behind the maps (boxes 64 x 128 for A, 64 x 32 for B over
// staging buffers of 7 * 64 elements per row/column) and their scales
// scaleA[a_row0 + i], scaleB[b_col0 + j].  C: FP64, any alignment.
// lshift >= 0: only the elements (i, j) with i >= j + lshift are written and
// sub-tiles wholly above that diagonal are skipped (the symmetric update of
// the Cholesky factorization, where B is L21^T staged like A).
cudaError_t launch_gemm_f64emu(int m, int n, const CUtensorMap &mapA, int a_row0, const CUtensorMap &mapB, int b_col0,
                               double *C, int ldc, const double *scaleA, const double *scaleB, int *tile_ctr, int *status,
                               long long bound_ns, int max_ctas, cudaStream_t s, CtaTrace tr, int lshift, SmShare sh,
                               int tile) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    if (sh.req && !sh.mask) return cudaErrorInvalidValue;
    int sms = 0;
    cudaError_t e = lu_sm_count(&sms);
    if (e != cudaSuccess) return e;
    // set on every launch: the attribute belongs to the current device's context
    e = cudaFuncSetAttribute(gemm_update_f64emu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEmSmem);
    if (e != cudaSuccess) return e;
    const long long mt = lu_ceil_div(m, kEmBM);
    // sub-tiles per task: tile 1: kEmMaxSub; 2: two; 0: fewer while the queue would not fill
    // the GPU twice (the task shape changes the schedule, not the arithmetic)
    int nsub = tile == 2 ? 2 : kEmMaxSub;
    if (tile == 0)
        while (nsub > 1 && mt * lu_ceil_div(n, (long long)kEmBN * nsub) < 2LL * sms) nsub >>= 1;
    const long long ntasks = mt * lu_ceil_div(n, (long long)kEmBN * nsub);
    const int cap = max_ctas > 0 && max_ctas < sms ? max_ctas : sms;
    int grid = (int)(ntasks < cap ? ntasks : cap);
    if (sh.mode == 1) grid = sh.join_ctas > 0 ? sh.join_ctas : 1;   // joins a running update: same counter
    if (sh.mode == 0) {
        cudaError_t ez = cudaMemsetAsync(tile_ctr, 0, sizeof(int), s);
        if (ez != cudaSuccess) return ez;
    }
    gemm_update_f64emu<<<grid, kEmThreads, kEmSmem, s>>>(m, n, mapA, a_row0, mapB, b_col0, C, ldc, scaleA, scaleB, nsub,
                                                          lshift, tile_ctr, status, bound_ns, tr, sh.req, sh.mask);
    lu_count_launch();
    return cudaGetLastError();
}

cudaError_t launch_stage_rows_f64emu(int rows, int k, const double *L, int ld, __nv_bfloat16 *stage, int lds, double *scale,
                                     cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    const int grid = lu_ceil_div(rows, 8) < 152 * 16 ? lu_ceil_div(rows, 8) : 152 * 16;
    stage_rows_f64emu<<<grid, 256, 0, s>>>(rows, k, kEmK, L, ld, stage, lds, scale);
    lu_count_launch();
    return cudaGetLastError();
}

cudaError_t launch_stage_cols_f64emu(int k, int cols, const double *B, int ld, __nv_bfloat16 *stage, int lds, double *scale,
                                     cudaStream_t s) {
    if (cols <= 0) return cudaSuccess;
    const int grid = lu_ceil_div(cols, 8) < 152 * 16 ? lu_ceil_div(cols, 8) : 152 * 16;
    stage_cols_f64emu<<<grid, 256, 0, s>>>(k, kEmK, cols, B, ld, stage, lds, scale);
    lu_count_launch();
    return cudaGetLastError();
}

}  // namespace lu
