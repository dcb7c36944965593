// Trailing update RL3 / PF2 / RU2 (section 3.1, Figure 1 right; section 3.2,
// Figure 3) on the 5th-generation tensor cores: C := C - A * B with C in FP32
// and the operands A = L21 and B = U12 rounded to BF16 (or split into two
// BF16 halves, three products), or to FP8 e4m3 with a power-of-two scale per
// staged row of A and per staged column of B (the epilogue multiplies the
// FP32 accumulator by the two exact reciprocal scales).
//
// Persistent, warp-specialized kernel, one CTA per SM, 128 x 128 tiles of C
// taken from a global atomic tile queue; all data movement through TMA:
//   warp 0   producer: tile index from the queue; the tile's C block (FP32,
//            128 rows x 128 columns, four 128 x 32 boxes) into the C buffer
//            once the previous tile's store has drained it; the K chunks of
//            the A and B tiles (128-byte swizzle) into a ring of stages;
//   warp 1   MMA issuer: tcgen05.mma kind::f16 (M=128, N=128, K=16) or
//            kind::f8f6f4 (K=32) into one
//            of two TMEM accumulators; tcgen05.commit frees stages and hands
//            the accumulator to the epilogue;
//   warps 2-5 epilogue: tcgen05.ld of the accumulator, C := C - acc in shared
//            memory, then a TMA store of each 128 x 32 box.
// So the HBM traffic of the update -- C read and written once in FP32 -- is
// carried by TMA and overlaps the MMAs of the same and the next tile.  Every
// mbarrier wait is bounded; on expiry the kernel records LU_ERR_TIMEOUT, waits
// once more (bounded) for its own copies, frees its TMEM and returns.
//
// Operand staging (K contiguous, K padded with zeros to one 128-byte swizzle
// span: 64 BF16 or 128 FP8 elements):
//   A: row-major, element (i, k) at stageA[i * lds + k]  (the panel's L21)
//   B: column-major, element (k, j) at stageB[j * lds + k]  (U12 by columns)
// With the split, the low halves follow at k + kpad.  FP8 staging carries
// scaleA[i] (= 2^-e_i, the inverse of the factor applied to row i) and
// scaleB[j].
#include "common.cuh"
#include "internal.h"
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include "tcgen05.cuh"

namespace lu {

constexpr int kTcBM = 128;
constexpr int kTcBN = 128;
constexpr int kTcBK = 64;            // one 128-byte swizzle span of BF16
constexpr int kTcBK8 = 128;          // one 128-byte swizzle span of FP8
constexpr int kTcMaxK = 256;
constexpr int kTcThreads = 192;      // 6 warps: TMA, MMA, 4 x epilogue
constexpr int kTcChunkA = kTcBM * kTcBK * 2;   // 16 KB
constexpr int kTcChunkB = kTcBN * kTcBK * 2;   // 16 KB
constexpr int kTcCBox = 32;                    // columns per C box
constexpr int kTcCBytes = kTcBM * kTcBN * 4;   // 64 KB C buffer
constexpr size_t kTcSmem = 1024 + (size_t)4 * (kTcChunkA + kTcChunkB) + kTcCBytes + 256;   // 4 x1 or 2 x3 stages

// NPROD: 1 = BF16, 3 = split BF16 (three products), 8 = FP8 e4m3 with scales.
template <int NPROD>
__global__ void __launch_bounds__(kTcThreads, 1)
gemm_update_tc(int m, int n, int K, const __grid_constant__ CUtensorMap mapA, int a_row0,
               const __grid_constant__ CUtensorMap mapB, int b_col0, const __grid_constant__ CUtensorMap mapC,
               int *__restrict__ tile_ctr, int *__restrict__ status, long long bound_ns,
               const float *__restrict__ scaleA, const float *__restrict__ scaleB, CtaTrace tr,
               const int *__restrict__ yreq, const unsigned *__restrict__ ymask) {
    const unsigned long long t_start = tr.ring ? lu_globaltimer() : 0ull;
    constexpr bool FP8 = NPROD == 8;
    constexpr int BK = FP8 ? kTcBK8 : kTcBK;        // K elements per 128-byte chunk
    constexpr int NSPLIT = NPROD == 3 ? 2 : 1;
    constexpr uint32_t kStageBytes = (uint32_t)NSPLIT * (kTcChunkA + kTcChunkB);
    constexpr int kStages = NSPLIT == 1 ? 4 : 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (base - raw);
    const uint32_t sC = base + (uint32_t)kStages * kStageBytes;          // C buffer, 4 boxes [32 cols][128 rows]
    float *Cs = reinterpret_cast<float *>(gbase + (size_t)kStages * kStageBytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + (size_t)kStages * kStageBytes + kTcCBytes);
    // bars: full[kStages], empty[kStages], acc_full[2], acc_empty[2], tile_full[2], c_full, c_empty
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8u * kStages;
    const uint32_t accf0 = empty0 + 8u * kStages, acce0 = accf0 + 16u, tilef0 = acce0 + 16u;
    const uint32_t cfull = tilef0 + 16u, cempty = cfull + 8u;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * kStages + 8);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *stage_tile = reinterpret_cast<volatile int *>(tmem_slot + 2);        // [kStages]
    volatile int *acc_tile = reinterpret_cast<volatile int *>(tmem_slot + 2 + kStages);  // [2]
    volatile int *ntiles_done = reinterpret_cast<volatile int *>(tmem_slot + 4 + kStages);  // tiles this CTA took

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nk = K / BK;                          // K is a multiple of BK
    const int kpad_off = K;                         // lo halves start at x = K
    const int mt = (m + kTcBM - 1) / kTcBM, ntl = (n + kTcBN - 1) / kTcBN;
    const int ntiles = mt * ntl;

    // a CTA that starts after the queue ran dry (the tail of a joining grid), or on
    // an SM the panel branch asked back, leaves before claiming TMEM
    __shared__ int leave;
    if (tid == 0) leave = *reinterpret_cast<volatile int *>(tile_ctr) >= ntiles || lu_share_yield(yreq, ymask);
    __syncthreads();
    if (leave) {
        if (tid == 0) lu_trace_cta(tr, t_start, 0);
        return;
    }

    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) { mbar_init(full0 + 8u * i, 1); mbar_init(empty0 + 8u * i, 1); }
        for (int i = 0; i < 2; ++i) {
            mbar_init(accf0 + 8u * i, 1);
            mbar_init(acce0 + 8u * i, 128);
            mbar_init(tilef0 + 8u * i, 1);
        }
        mbar_init(cfull, 1);
        mbar_init(cempty, 1);
        *abort_flag = 0;
        *ntiles_done = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * kTcBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0, cph = 0;
            for (;;) {
                // worker sharing: on the panel's SMs, stop at a tile boundary when asked
                int t = lu_share_yield(yreq, ymask) ? -1 : atomicAdd(tile_ctr, 1);
                if (t >= ntiles || *abort_flag) t = -1;
                if (t >= 0) *ntiles_done = *ntiles_done + 1;
                const int tm = t >= 0 ? (t % mt) * kTcBM : 0, tn = t >= 0 ? (t / mt) * kTcBN : 0;
                bool ok = true;
                const int chunks = t >= 0 ? nk : 1;
                for (int kc = 0; kc < chunks && ok; ++kc) {
                    if (!mbar_wait_bounded(empty0 + 8u * s, ph ^ 1u, bound_ns)) { *abort_flag = 1; ok = false; break; }
                    const uint32_t st = base + (uint32_t)s * kStageBytes;
                    const uint32_t fb = full0 + 8u * s;
                    stage_tile[s] = t;
                    if (t < 0) {
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(fb) : "memory");
                    } else {
                        mbar_expect_tx(fb, kStageBytes);
                        tma_load_2d(st, &mapA, kc * BK, a_row0 + tm, fb);
                        tma_load_2d(st + NSPLIT * kTcChunkA, &mapB, kc * BK, b_col0 + tn, fb);
                        if (NSPLIT == 2) {
                            tma_load_2d(st + kTcChunkA, &mapA, kpad_off + kc * BK, a_row0 + tm, fb);
                            tma_load_2d(st + 2 * kTcChunkA + kTcChunkB, &mapB, kpad_off + kc * BK, b_col0 + tn, fb);
                        }
                    }
                    if (++s == kStages) { s = 0; ph ^= 1u; }
                }
                // the tile's C block, once the previous tile's store has left the buffer
                if (t >= 0 && ok) {
                    if (!mbar_wait_bounded(cempty, cph ^ 1u, bound_ns)) { *abort_flag = 1; ok = false; }
                    else {
                        mbar_expect_tx(cfull, (uint32_t)kTcCBytes);
#pragma unroll
                        for (int b = 0; b < kTcBN / kTcCBox; ++b)
                            tma_load_2d(sC + (uint32_t)b * (kTcBM * kTcCBox * 4), &mapC, tm, tn + b * kTcCBox, cfull);
                        cph ^= 1u;
                    }
                }
                if (t < 0 || !ok) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = FP8 ? umma_idesc_e4m3(kTcBM, kTcBN) : umma_idesc_bf16(kTcBM, kTcBN);
            int s = 0;
            uint32_t ph = 0;
            for (int it = 0;; ++it) {
                const int a = it & 1;
                const uint32_t aph = (uint32_t)((it >> 1) & 1);
                // the accumulator must be free before its tile index is replaced
                bool stop = false;
                if (!mbar_wait_bounded(acce0 + 8u * a, aph ^ 1u, bound_ns)) { *abort_flag = 1; stop = true; }
                if (*abort_flag) stop = true;
                int t = -1;
                if (!stop) {
                    if (!mbar_wait_bounded(full0 + 8u * s, ph, bound_ns)) { *abort_flag = 1; stop = true; }
                    else t = stage_tile[s];
                }
                if (stop || t < 0) {
                    acc_tile[a] = -1;
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tilef0 + 8u * a) : "memory");
                    break;
                }
                acc_tile[a] = t;
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tilef0 + 8u * a) : "memory");
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem + (uint32_t)(a * kTcBN);
                bool ok = true;
                for (int kc = 0; kc < nk; ++kc) {
                    if (kc > 0 && !mbar_wait_bounded(full0 + 8u * s, ph, bound_ns)) { *abort_flag = 1; ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t st = base + (uint32_t)s * kStageBytes;
                    const uint32_t sAh = st, sAl = st + kTcChunkA;
                    const uint32_t sBh = st + NSPLIT * kTcChunkA, sBl = sBh + kTcChunkB;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {   // four MMAs of 32 bytes of K per 128-byte chunk
                        const uint32_t first = (kc | kk) == 0 ? 0u : 1u;
                        if (FP8)
                            umma_e4m3(acc, umma_desc_sw128(sAh + kk * 32), umma_desc_sw128(sBh + kk * 32), idesc, first);
                        else
                            umma_bf16(acc, umma_desc_sw128(sAh + kk * 32), umma_desc_sw128(sBh + kk * 32), idesc, first);
                        if (NPROD == 3) {
                            umma_bf16(acc, umma_desc_sw128(sAh + kk * 32), umma_desc_sw128(sBl + kk * 32), idesc, 1u);
                            umma_bf16(acc, umma_desc_sw128(sAl + kk * 32), umma_desc_sw128(sBh + kk * 32), idesc, 1u);
                        }
                    }
                    umma_commit(empty0 + 8u * s);            // stage free once these MMAs are done
                    if (++s == kStages) { s = 0; ph ^= 1u; }
                }
                if (!ok) {
                    // the epilogue of this tile is already waiting: release it without data
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(accf0 + 8u * a) : "memory");
                    break;
                }
                umma_commit(accf0 + 8u * a);                 // accumulator ready
            }
        }
    } else {
        // epilogue: warps 2..5 own TMEM lane quarters (warp % 4); thread = tile row
        const int q = warp & 3;
        const int r = q * 32 + lane;
        const bool leader = (tid == 64);
        uint32_t cph = 0;
        for (int it = 0;; ++it) {
            const int a = it & 1;
            const uint32_t aph = (uint32_t)((it >> 1) & 1);
            if (!mbar_wait_bounded(tilef0 + 8u * a, aph, bound_ns)) { *abort_flag = 1; break; }
            const int t = acc_tile[a];
            if (t < 0) break;
            const int tm = (t % mt) * kTcBM, tn = (t / mt) * kTcBN;
            bool ok = mbar_wait_bounded(cfull, cph, bound_ns) && mbar_wait_bounded(accf0 + 8u * a, aph, bound_ns);
            cph ^= 1u;
            if (!ok || *abort_flag) { *abort_flag = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc = tmem + (uint32_t)(a * kTcBN) + ((uint32_t)(q * 32) << 16);
            // FP8: undo the staging scales (powers of two: exact)
            const float sa = FP8 ? (tm + r < m ? scaleA[a_row0 + tm + r] : 0.f) : 1.f;
#pragma unroll
            for (int h = 0; h < kTcBN / 32; ++h) {
                float v[32];
                tmem_ld32(acc + (uint32_t)(h * 32), v);
                float *box = Cs + (size_t)h * (kTcBM * kTcCBox);   // box h: [32 cols][128 rows]
                if (FP8) {
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        const int col = tn + h * 32 + c;
                        const float sb = col < n ? __ldg(&scaleB[b_col0 + col]) : 0.f;
                        box[c * kTcBM + r] -= v[c] * sa * sb;
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 32; ++c) box[c * kTcBM + r] -= v[c];
                }
            }
            // accumulator read: the MMAs of the tile after next may start
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce0 + 8u * a) : "memory");
            // results visible to the async proxy, then one thread stores the boxes
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if (leader) {
#pragma unroll
                for (int b = 0; b < kTcBN / kTcCBox; ++b)
                    tma_store_2d(&mapC, tm, tn + b * kTcCBox, sC + (uint32_t)b * (kTcBM * kTcCBox * 4));
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(cempty) : "memory");
            }
        }
        if (leader) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0 && *abort_flag) {
        atomicExch(status, (int)LU_ERR_TIMEOUT);
        // give copies in flight one bounded chance to land before shared memory is released
        for (int i = 0; i < kStages; ++i) mbar_wait_bounded(full0 + 8u * i, 0, bound_ns / 4);
        mbar_wait_bounded(cfull, 0, bound_ns / 4);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTcBN) : "memory");
    }
    if (tid == 0) lu_trace_cta(tr, t_start, *ntiles_done);
}

// ---- operand staging -------------------------------------------------------

// L21 (rows x k, FP32 column-major, ld) -> BF16 row-major stage[i * lds + kk],
// zero for kk in [k, kpad); with split, the low part x - bf16(x) rounded to
// BF16 goes to stage[i * lds + kpad + kk].  Tiles of 32 x 32 transposed through
// shared memory.
__global__ void stage_rows_bf16(int rows, int k, int kpad, const float *__restrict__ L, int ld,
                                __nv_bfloat16 *__restrict__ stage, int lds, int split) {
    __shared__ float t[32][33];
    const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    for (int yy = ty; yy < 32; yy += 8) {
        const int i = i0 + tx, kk = k0 + yy;
        t[yy][tx] = (i < rows && kk < k) ? L[(size_t)i + (size_t)kk * ld] : 0.f;
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
        const int i = i0 + yy, kk = k0 + tx;
        if (i < rows && kk < kpad) {
            const float x = t[tx][yy];
            const __nv_bfloat16 hi = __float2bfloat16_rn(x);
            stage[(size_t)i * lds + kk] = hi;
            if (split) stage[(size_t)i * lds + kpad + kk] = __float2bfloat16_rn(x - __bfloat162float(hi));
        }
    }
}

// B (k x cols, FP32 column-major, ld) -> BF16 stage[j * lds + kk], zero pad.
__global__ void stage_cols_bf16(int k, int kpad, int cols, const float *__restrict__ B, int ld,
                                __nv_bfloat16 *__restrict__ stage, int lds, int split) {
    const size_t total = (size_t)cols * kpad;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int kk = (int)(e % kpad), j = (int)(e / kpad);
        const float x = kk < k ? B[(size_t)kk + (size_t)j * ld] : 0.f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        stage[(size_t)j * lds + kk] = hi;
        if (split) stage[(size_t)j * lds + kpad + kk] = __float2bfloat16_rn(x - __bfloat162float(hi));
    }
}

// L21 (rows x k, FP32 column-major) -> e4m3 row-major stage[i * lds + kk], one
// power-of-two scale per row: scale[i] = the inverse multiplier.  One warp per row.
__global__ void stage_rows_fp8(int rows, int k, int kpad, const float *__restrict__ L, int ld,
                               unsigned char *__restrict__ stage, int lds, float *__restrict__ scale) {
    const int lane = threadIdx.x & 31;
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < rows; i += gridDim.x * (blockDim.x >> 5)) {
        float amax = 0.f;
        for (int kk = lane; kk < k; kk += 32) amax = fmaxf(amax, fabsf(L[(size_t)i + (size_t)kk * ld]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        float inv;
        const float mul = lu_fp8_scale(amax, &inv);
        if (lane == 0) scale[i] = inv;
        for (int kk = lane; kk < kpad; kk += 32)
            stage[(size_t)i * lds + kk] = kk < k ? lu_to_e4m3(L[(size_t)i + (size_t)kk * ld] * mul) : (unsigned char)0;
    }
}

// B (k x cols, FP32 column-major) -> e4m3 stage[j * lds + kk], one scale per column.
__global__ void stage_cols_fp8(int k, int kpad, int cols, const float *__restrict__ B, int ld,
                               unsigned char *__restrict__ stage, int lds, float *__restrict__ scale) {
    const int lane = threadIdx.x & 31;
    for (int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < cols; j += gridDim.x * (blockDim.x >> 5)) {
        float amax = 0.f;
        for (int kk = lane; kk < k; kk += 32) amax = fmaxf(amax, fabsf(B[(size_t)kk + (size_t)j * ld]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        float inv;
        const float mul = lu_fp8_scale(amax, &inv);
        if (lane == 0) scale[j] = inv;
        for (int kk = lane; kk < kpad; kk += 32)
            stage[(size_t)j * lds + kk] = kk < k ? lu_to_e4m3(B[(size_t)kk + (size_t)j * ld] * mul) : (unsigned char)0;
    }
}

// ---- host side ---------------------------------------------------------------

// 2-D map over a K-major staging buffer (BF16, or FP8 bytes when fp8): inner
// dimension kinner elements, outer dimension `outer` rows/columns, leading
// dimension lds elements; boxes of one 128-byte swizzle span x box_outer.
cudaError_t make_stage_map(CUtensorMap *map, const void *base, int kinner, int outer, int lds, int box_outer, int fp8) {
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    const int esz = fp8 ? 1 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)kinner, (cuuint64_t)(outer > 0 ? outer : 1)};
    cuuint64_t strides[1] = {(cuuint64_t)lds * esz};
    cuuint32_t box[2] = {(cuuint32_t)(fp8 ? kTcBK8 : kTcBK), (cuuint32_t)box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode.load()(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                          const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// kinner: elements per staged row/column (kpad, or 2 kpad when split)
cudaError_t make_stage_maps(CUtensorMap *mapA, const void *stageA, int rowsA, CUtensorMap *mapB, const void *stageB,
                            int colsB, int kinner, int lds, int fp8) {
    cudaError_t e = make_stage_map(mapA, stageA, kinner, rowsA, lds, kTcBM, fp8);
    if (e != cudaSuccess) return e;
    return make_stage_map(mapB, stageB, kinner, colsB, lds, kTcBN, fp8);
}

int tc_box_rows() { return kTcBM; }
int tc_box_cols() { return kTcBN; }

// 2-D FP32 map over the m x n column-major block at C (leading dimension ldc):
// x = row (contiguous), y = column; boxes of 128 rows x 32 columns.  TMA needs
// C 16-byte aligned and ldc a multiple of 4 (checked by the caller).
static cudaError_t make_c_map(CUtensorMap *map, float *C, int m, int n, int ldc) {
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)ldc * 4};
    cuuint32_t box[2] = {(cuuint32_t)kTcBM, (cuuint32_t)kTcCBox};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode.load()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, C, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

bool tc_c_aligned(const float *C, int ldc) { return ((uintptr_t)C % 16 == 0) && (ldc % 4 == 0); }

template <int NPROD>
static cudaError_t launch_tc_mode(int grid, int m, int n, int K, const CUtensorMap &mapA, int a_row0, const CUtensorMap &mapB,
                                  int b_col0, const CUtensorMap &mapC, int *tile_ctr, int *status, long long bound_ns,
                                  const float *scaleA, const float *scaleB, cudaStream_t s, const CtaTrace &tr,
                                  const SmShare &sh) {
    // set on every launch: the attribute belongs to the current device's context
    cudaError_t e = cudaFuncSetAttribute(gemm_update_tc<NPROD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e != cudaSuccess) return e;
    gemm_update_tc<NPROD><<<grid, kTcThreads, kTcSmem, s>>>(m, n, K, mapA, a_row0, mapB, b_col0, mapC, tile_ctr, status,
                                                             bound_ns, scaleA, scaleB, tr, sh.req, sh.mask);
    lu_count_launch();
    return cudaGetLastError();
}

// C[m x n] -= A[a_row0 + (0..m), 0..K) * B[0..K, b_col0 + (0..n)] through the maps
// (nprod = 1: BF16 operands; 3: split BF16, staging holds hi | lo; 8: FP8 e4m3
// with the row scales scaleA[a_row0 + i] and column scales scaleB[b_col0 + j]).
// C must be 16-byte aligned with ldc a multiple of 4 (tc_c_aligned).
cudaError_t launch_gemm_tc(int nprod, int m, int n, int K, const CUtensorMap &mapA, int a_row0, const CUtensorMap &mapB,
                           int b_col0, float *C, int ldc, int *tile_ctr, int *status, long long bound_ns, cudaStream_t s,
                           const float *scaleA, const float *scaleB, int max_ctas, CtaTrace tr, SmShare sh) {
    if (m <= 0 || n <= 0 || K <= 0) return cudaSuccess;
    if (sh.req && !sh.mask) return cudaErrorInvalidValue;
    if (nprod != 1 && nprod != 3 && nprod != 8) return cudaErrorInvalidValue;
    const int bk = nprod == 8 ? kTcBK8 : kTcBK;
    if (K > (nprod == 8 ? 2 * kTcMaxK : kTcMaxK) || K % bk != 0) return cudaErrorInvalidValue;
    if (nprod == 8 && (!scaleA || !scaleB)) return cudaErrorInvalidValue;
    if (!tc_c_aligned(C, ldc)) return cudaErrorInvalidValue;
    CUtensorMap mapC;
    cudaError_t ec = make_c_map(&mapC, C, m, n, ldc);
    if (ec != cudaSuccess) return ec;
    int sms = 0;
    ec = lu_sm_count(&sms);
    if (ec != cudaSuccess) return ec;
    const int ntiles = lu_ceil_div(m, kTcBM) * lu_ceil_div(n, kTcBN);
    // persistent CTAs: one per SM, or max_ctas (> 0) to leave SMs to other work
    const int cap = max_ctas > 0 && max_ctas < sms ? max_ctas : sms;
    int grid = ntiles < cap ? ntiles : cap;
    if (sh.mode == 1) grid = sh.join_ctas > 0 ? sh.join_ctas : 1;   // joins a running update: same counter
    if (sh.mode == 0) {
        cudaError_t ez = cudaMemsetAsync(tile_ctr, 0, sizeof(int), s);
        if (ez != cudaSuccess) return ez;
    }
    if (nprod == 1) return launch_tc_mode<1>(grid, m, n, K, mapA, a_row0, mapB, b_col0, mapC, tile_ctr, status, bound_ns, nullptr, nullptr, s, tr, sh);
    if (nprod == 3) return launch_tc_mode<3>(grid, m, n, K, mapA, a_row0, mapB, b_col0, mapC, tile_ctr, status, bound_ns, nullptr, nullptr, s, tr, sh);
    return launch_tc_mode<8>(grid, m, n, K, mapA, a_row0, mapB, b_col0, mapC, tile_ctr, status, bound_ns, scaleA, scaleB, s, tr, sh);
}

cudaError_t launch_stage_rows(int rows, int k, int kpad, const float *L, int ld, __nv_bfloat16 *stage, int lds, int split,
                              cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    dim3 grid(lu_ceil_div(rows, 32), lu_ceil_div(kpad, 32));
    stage_rows_bf16<<<grid, 256, 0, s>>>(rows, k, kpad, L, ld, stage, lds, split);
    lu_count_launch();
    return cudaGetLastError();
}

cudaError_t launch_stage_cols(int k, int kpad, int cols, const float *B, int ld, __nv_bfloat16 *stage, int lds, int split,
                              cudaStream_t s) {
    if (cols <= 0) return cudaSuccess;
    size_t total = (size_t)cols * kpad;
    int grid = (int)((total + 255) / 256 < 152 * 16 ? (total + 255) / 256 : 152 * 16);
    stage_cols_bf16<<<grid, 256, 0, s>>>(k, kpad, cols, B, ld, stage, lds, split);
    lu_count_launch();
    return cudaGetLastError();
}

cudaError_t launch_stage_rows_fp8(int rows, int k, int kpad, const float *L, int ld, unsigned char *stage, int lds,
                                  float *scale, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    const int grid = lu_ceil_div(rows, 8) < 152 * 16 ? lu_ceil_div(rows, 8) : 152 * 16;
    stage_rows_fp8<<<grid, 256, 0, s>>>(rows, k, kpad, L, ld, stage, lds, scale);
    lu_count_launch();
    return cudaGetLastError();
}

cudaError_t launch_stage_cols_fp8(int k, int kpad, int cols, const float *B, int ld, unsigned char *stage, int lds,
                                  float *scale, cudaStream_t s) {
    if (cols <= 0) return cudaSuccess;
    const int grid = lu_ceil_div(cols, 8) < 152 * 16 ? lu_ceil_div(cols, 8) : 152 * 16;
    stage_cols_fp8<<<grid, 256, 0, s>>>(k, kpad, cols, B, ld, stage, lds, scale);
    lu_count_launch();
    return cudaGetLastError();
}

// K padded to whole 128-byte chunks: 64 BF16 or 128 FP8 elements
int tc_kpad(int k, int fp8) {
    const int bk = fp8 ? kTcBK8 : kTcBK;
    return ((k + bk - 1) / bk) * bk;
}
int tc_max_k() { return kTcMaxK; }

}  // namespace lu
