// Panel factorization (RL1 / PF3 of the paper) on one thread-block cluster.
//
// Section 3.1, Figure 1 (left): unblocked right-looking LU of the m x W panel
// with partial pivoting -- per column j: pivot search over rows j..m-1, row
// interchange, a21 := a21 / alpha11, A22 := A22 - a21 a12^T.  The paper
// stresses that this step has little concurrency and sits on the critical
// path (section 3.1, Figure 2); here the panel's rows are spread over the
// shared memory of the CTAs of one cluster (up to 16 SMs), so each column step
// costs one hardware cluster barrier:
//
//   1. every CTA reduces the (|a|, row) maximum of its rows (warp shuffles,
//      then shared memory), and publishes that candidate row and, for the CTA
//      holding row j, row j itself into a double-buffered slot;
//   2. barrier.cluster;
//   3. every CTA reads the candidates of all CTAs through distributed shared
//      memory, picks the winner (largest magnitude, smallest row on ties), takes
//      the pivot row from the winner's slot, and the two owners write the
//      interchanged rows locally;
//   4. every CTA scales its part of column j (IEEE division) and applies the
//      rank-1 update to its rows, tracking the candidate of column j+1.
//
// The interchanges are applied to the panel's W columns only; the other
// columns are handled by the row-interchange kernel (swap_trsm.cu).
#include "common.cuh"
#include <cooperative_groups.h>
#include <climits>

namespace cg = cooperative_groups;

namespace lu {

constexpr int kPanelThreads = 512;
constexpr int kPanelWMax = 64;

template <typename T>
struct PanelSlot {
    T mag;                  // candidate |value| (-1: no candidate)
    int row;                // panel-local candidate row (INT_MAX: none)
    int pad;
    T cand[kPanelWMax];     // candidate row, all W columns
    T diag[kPanelWMax];     // row j, published by its owner
};

template <typename T>
__device__ __forceinline__ void warp_argmax(T &mag, int &idx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T m2 = __shfl_xor_sync(0xffffffffu, mag, o);
        int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        if (lu_better(m2, i2, mag, idx)) { mag = m2; idx = i2; }
    }
}

size_t panel_smem_bytes(int R, int W, size_t elem) {
    size_t a = (size_t)R * W * elem;
    a = (a + 15) & ~(size_t)15;
    size_t slot = (elem == 8) ? sizeof(PanelSlot<double>) : sizeof(PanelSlot<float>);
    a += 2 * slot;
    a += 2 * kPanelWMax * elem;          // urow, drow
    a += 32 * (elem + sizeof(int));      // warp candidates
    a += 16 * sizeof(int);               // broadcast words
    return a + 64;
}

// P: top-left of the panel (rows 0..m-1 of the panel, columns 0..W-1), leading
// dimension lda.  Rows are split into blocks of R per CTA (cluster rank order).
// ipiv: ipiv entries of this panel (W of them), written as row_base + p + 1.
// info: first zero pivot as row_base + j + 1 (only if *info is still 0).
template <typename T>
__global__ void __launch_bounds__(kPanelThreads, 1)
panel_getf2_cluster(T *__restrict__ P, int lda, int m, int W, int R, int *__restrict__ ipiv,
                    int row_base, int *__restrict__ info) {
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = kPanelThreads / 32;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *As = reinterpret_cast<T *>(smem_raw);
    size_t off = ((size_t)R * W * sizeof(T) + 15) & ~(size_t)15;
    PanelSlot<T> *slots = reinterpret_cast<PanelSlot<T> *>(smem_raw + off);
    T *urow = reinterpret_cast<T *>(slots + 2);
    T *drow = urow + kPanelWMax;
    T *red_mag = drow + kPanelWMax;
    int *red_idx = reinterpret_cast<int *>(red_mag + 32);
    int *bc = red_idx + 32;

    const int r0 = rank * R;
    const int myR = max(0, min(R, m - r0));

    // load this CTA's rows of the panel (coalesced down each column)
    for (int c = 0; c < W; ++c)
        for (int lr = tid; lr < myR; lr += kPanelThreads)
            As[(size_t)c * R + lr] = P[(size_t)(r0 + lr) + (size_t)c * lda];
    __syncthreads();

    // candidate for column 0
    T best = T(-1);
    int bidx = INT_MAX;
    for (int lr = tid; lr < myR; lr += kPanelThreads) {
        T v = lu_abs(As[lr]);
        if (lu_better(v, r0 + lr, best, bidx)) { best = v; bidx = r0 + lr; }
    }

    const int kmax = min(m, W);
    for (int j = 0; j < kmax; ++j) {
        PanelSlot<T> *slot = &slots[j & 1];
        // (1) CTA-level argmax, publish
        warp_argmax(best, bidx);
        if (lane == 0) { red_mag[warp] = best; red_idx[warp] = bidx; }
        __syncthreads();
        if (warp == 0) {
            T mg = lane < nwarps ? red_mag[lane] : T(-1);
            int ix = lane < nwarps ? red_idx[lane] : INT_MAX;
            warp_argmax(mg, ix);
            if (lane == 0) { slot->mag = mg; slot->row = ix; }
        }
        __syncthreads();
        const int crow = slot->row;
        if (tid < W) {
            if (crow != INT_MAX) slot->cand[tid] = As[(size_t)tid * R + (crow - r0)];
            if (j >= r0 && j < r0 + myR) slot->diag[tid] = As[(size_t)tid * R + (j - r0)];
        }
        // (2) one hardware cluster barrier per column (release / acquire)
        cl.sync();
        // (3) winner over the cluster through distributed shared memory
        if (warp == 0) {
            T mg = T(-1);
            int ix = INT_MAX;
            if (lane < C) {
                PanelSlot<T> *rs = cl.map_shared_rank(slot, lane);
                mg = rs->mag;
                ix = rs->row;
            }
            warp_argmax(mg, ix);
            if (lane == 0) bc[0] = ix;
        }
        __syncthreads();
        int p = bc[0];
        const bool valid = (p != INT_MAX);
        if (!valid) p = j;   // every candidate NaN: keep row j, as a sequential scan would
        const int owner_j = j / R;
        const int owner_p = p / R;
        if (tid < W) {
            PanelSlot<T> *sp = cl.map_shared_rank(&slots[j & 1], valid ? owner_p : owner_j);
            urow[tid] = valid ? sp->cand[tid] : sp->diag[tid];
            if (p != j) {
                PanelSlot<T> *sj = cl.map_shared_rank(&slots[j & 1], owner_j);
                drow[tid] = sj->diag[tid];
            }
        }
        __syncthreads();
        const T piv = urow[j];
        const bool zero = (piv == T(0));
        if (!zero && p != j && tid < W) {
            if (rank == owner_p) As[(size_t)tid * R + (p - r0)] = drow[tid];
            if (rank == owner_j) As[(size_t)tid * R + (j - r0)] = urow[tid];
        }
        if (rank == 0 && tid == 0) {
            ipiv[j] = row_base + p + 1;
            if (zero) atomicCAS(info, 0, row_base + j + 1);
        }
        __syncthreads();
        // (4) scale and rank-1 update of this CTA's rows below j; next candidate
        best = T(-1);
        bidx = INT_MAX;
        const bool has_next = (j + 1 < W);
        for (int lr = tid; lr < myR; lr += kPanelThreads) {
            const int i = r0 + lr;
            if (i <= j) continue;
            if (!zero) {
                const T l = As[(size_t)j * R + lr] / piv;
                As[(size_t)j * R + lr] = l;
                for (int c = j + 1; c < W; ++c) {
                    T *a = &As[(size_t)c * R + lr];
                    *a = fma(-l, urow[c], *a);
                }
            }
            if (has_next) {
                T v = lu_abs(As[(size_t)(j + 1) * R + lr]);
                if (lu_better(v, i, best, bidx)) { best = v; bidx = i; }
            }
        }
        __syncthreads();
    }

    // write the factored panel back
    for (int c = 0; c < W; ++c)
        for (int lr = tid; lr < myR; lr += kPanelThreads)
            P[(size_t)(r0 + lr) + (size_t)c * lda] = As[(size_t)c * R + lr];
    // no CTA may leave while another can still read its slots
    cl.sync();
}

// Host launcher.  Chooses the cluster size and rows per CTA so the panel fits
// in shared memory; returns cudaErrorInvalidValue when it cannot.
template <typename T>
cudaError_t launch_panel(T *P, int lda, int m, int W, int *ipiv, int row_base, int *info,
                         int max_ctas, size_t smem_cap, cudaStream_t s) {
    if (W > kPanelWMax || W <= 0 || m <= 0) return cudaErrorInvalidValue;
    auto rows_for = [&](int c) {
        int r = (m + c - 1) / c;
        return (r + 31) & ~31;
    };
    if (max_ctas < 1) max_ctas = 16;
    int C = 1;
    // parallelism target: about one row per thread, at most max_ctas CTAs
    while (C < 16 && C < max_ctas && rows_for(C) > kPanelThreads) C *= 2;
    // capacity: the panel must fit in the cluster's shared memory
    while (C < 16 && panel_smem_bytes(rows_for(C), W, sizeof(T)) > smem_cap) C *= 2;
    if (C > 16) C = 16;
    int R = rows_for(C);
    if (panel_smem_bytes(R, W, sizeof(T)) > smem_cap) return cudaErrorInvalidValue;
    while (C > 1 && (long long)(C - 1) * R >= m) --C;   // no empty CTAs
    size_t smem = panel_smem_bytes(R, W, sizeof(T));
    cudaError_t e = cudaFuncSetAttribute(panel_getf2_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(panel_getf2_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(kPanelThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    lu_count_launch();
    return cudaLaunchKernelEx(&cfg, panel_getf2_cluster<T>, P, lda, m, W, R, ipiv, row_base, info);
}

// Largest panel width (power of two, <= cap) whose m rows fit in a 16-CTA cluster.
int panel_width_that_fits(int m, size_t elem, size_t smem_cap, int cap) {
    for (int W = cap; W >= 1; W >>= 1) {
        int R = (m + 15) / 16;
        R = (R + 31) & ~31;
        if (panel_smem_bytes(R, W, elem) <= smem_cap) return W;
    }
    return 0;
}

template cudaError_t launch_panel<double>(double *, int, int, int, int *, int, int *, int, size_t, cudaStream_t);
template cudaError_t launch_panel<float>(float *, int, int, int, int *, int, int *, int, size_t, cudaStream_t);

}  // namespace lu
