// Declarations shared between the library's translation units: each kernel
// launcher and internal entry point is declared here once, with its default
// arguments, and defined in the .cu file named above its group.
#pragma once
#include "common.cuh"
#include <cuda.h>
#include <cuda_bf16.h>

namespace lu {
// panel.cu
template <typename T>
cudaError_t launch_panel_outer(T *P, int lda, int m, int bo, int bi, int *ipiv, int row_base, int *info, int *map_out,
                               int *perm, StageDesc sd, int max_ctas, size_t smem_cap, int *status, long long bound_ns,
                               cudaStream_t s, CtaTrace tr, int *yreq, EtArgs et = EtArgs{});
cudaError_t launch_et_signal(int *flag, int epoch, cudaStream_t s);
int panel_width_that_fits(int m, size_t elem, size_t smem_cap, int cap, int bo);
int panel_cluster_ctas(int m, size_t elem, int bo, int bi, int max_ctas, size_t smem_cap);
cudaError_t launch_cluster_sm_probe(int C, unsigned *mask, cudaStream_t s);
cudaError_t launch_share_raise(int *req, cudaStream_t s);
bool panel_fits(int m, size_t elem, int bo, int bi, int max_ctas, size_t smem_cap);
// swap_trsm.cu
template <typename T>
cudaError_t launch_swap_trsm(T *A, int lda, int kb, int b, const int *map, int c_begin, int c_end, int do_trsm,
                             StageDesc sd, int stage_c0, cudaStream_t s, CtaTrace tr = CtaTrace{});
// gemm_simt.cu
template <typename T>
cudaError_t launch_gemm_simt(int m, int n, int k, const T *A, int lda, const T *B, int ldb, T *C, int ldc, cudaStream_t s,
                             CtaTrace tr = CtaTrace{}, bool transb = false, int lshift = -1, int tile = 0);
// gemm_tc.cu
cudaError_t make_stage_maps(CUtensorMap *mapA, const void *stageA, int rowsA, CUtensorMap *mapB, const void *stageB,
                            int colsB, int kinner, int lds, int fp8);
int tc_box_rows();
int tc_box_cols();
cudaError_t make_stage_map(CUtensorMap *map, const void *base, int kinner, int outer, int lds, int box_outer, int fp8);
cudaError_t launch_gemm_tc(int nprod, int m, int n, int K, const CUtensorMap &mapA, int a_row0, const CUtensorMap &mapB,
                           int b_col0, float *C, int ldc, int *tile_ctr, int *status, long long bound_ns, cudaStream_t s,
                           const float *scaleA, const float *scaleB, int max_ctas = 0, CtaTrace tr = CtaTrace{},
                           SmShare sh = SmShare{});
cudaError_t launch_stage_rows_fp8(int rows, int k, int kpad, const float *L, int ld, unsigned char *stage, int lds,
                                  float *scale, cudaStream_t s);
cudaError_t launch_stage_cols_fp8(int k, int kpad, int cols, const float *B, int ld, unsigned char *stage, int lds,
                                  float *scale, cudaStream_t s);
cudaError_t launch_stage_rows(int rows, int k, int kpad, const float *L, int ld, __nv_bfloat16 *stage, int lds, int split,
                              cudaStream_t s);
cudaError_t launch_stage_cols(int k, int kpad, int cols, const float *B, int ld, __nv_bfloat16 *stage, int lds, int split,
                              cudaStream_t s);
int tc_kpad(int k, int fp8);
int tc_max_k();
bool tc_c_aligned(const float *C, int ldc);
// gemm_f64emu.cu
cudaError_t launch_gemm_f64emu(int m, int n, const CUtensorMap &mapA, int a_row0, const CUtensorMap &mapB, int b_col0,
                               double *C, int ldc, const double *scaleA, const double *scaleB, int *tile_ctr, int *status,
                               long long bound_ns, int max_ctas, cudaStream_t s, CtaTrace tr = CtaTrace{},
                               int lshift = -1, SmShare sh = SmShare{}, int tile = 0);
cudaError_t launch_stage_rows_f64emu(int rows, int k, const double *L, int ld, __nv_bfloat16 *stage, int lds, double *scale,
                                     cudaStream_t s);
cudaError_t launch_stage_cols_f64emu(int k, int cols, const double *B, int ld, __nv_bfloat16 *stage, int lds, double *scale,
                                     cudaStream_t s);
int f64emu_kpad();
int f64emu_box_rows();
int f64emu_box_cols();
// solve.cu
cudaError_t launch_ipiv_to_perm(const int *ipiv, int n, int *perm, cudaStream_t s);
template <typename TI, typename TO>
cudaError_t launch_gather_rows(int n, int nrhs, const int *perm, const TI *B, int ldb, TO *X, int ldx, cudaStream_t s);
template <typename T>
cudaError_t launch_trsv_pair(const T *LU, int lda, int n, int nrhs, T *X, int ldx, int *ws, int *status, long long bound_ns,
                             int sms, cudaStream_t s, const T *Dinv = nullptr);
template <typename T>
cudaError_t launch_diag_inverse(const T *LU, int lda, int n, T *Dinv, cudaStream_t s);
template <typename T>
size_t trsv_inverse_elems(int n);
size_t trsv_workspace_ints(int n, int nrhs);
cudaError_t launch_trsv_timeout_selftest(const float *LU, int n, float *X, int *ws, int *status, long long bound_ns,
                                         cudaStream_t s);
cudaError_t launch_div_selftest(int dt64, long long count, unsigned long long seed, unsigned long long *mismatch,
                                cudaStream_t s);
cudaError_t launch_iota(int *v, int n, cudaStream_t s);
// batched_blocked.cu
constexpr int kBatchedBlockedMaxN = 256;
size_t batched_blocked_workspace_ints(int batch);
template <typename T>
cudaError_t launch_getrf_batched_blocked(int batch, const int *ns, T *const *As, const int *ldas, int *const *ipivs,
                                         int *infos, int nb, int *ws, int sms, cudaStream_t s);
template <typename T>
cudaError_t launch_getrs_batched_warp(int batch, int nrhs, const int *ns, const T *const *LUs, const int *ldas,
                                      const int *const *ipivs, T *const *Bs, const int *ldbs, int sms, cudaStream_t s);
// batched.cu
template <typename T>
cudaError_t launch_getrf_batched(int batch, const int *ns, T *const *As, const int *ldas, int *const *ipivs, int *infos,
                                 int max_n, cudaStream_t s);
template <typename T>
cudaError_t launch_getrs_batched(int batch, int nrhs, const int *ns, const T *const *LUs, const int *ldas,
                                 const int *const *ipivs, T *const *Bs, const int *ldbs, int max_n, cudaStream_t s);
// mixed.cu
cudaError_t launch_cast_rowsum(int n, const double *A, int lda, float *A32, int lda32, double *rowsum, cudaStream_t s);
size_t residual_workspace_doubles(int n, int nrhs);
cudaError_t launch_residual(int n, int nrhs, const double *A, int lda, const double *X, int ldx, const double *B, int ldb,
                            double *R, int ldr, double *part, unsigned long long *rmax, cudaStream_t s);
cudaError_t launch_absmax(int n, int nrhs, const double *V, int ldv, unsigned long long *out, cudaStream_t s);
cudaError_t launch_vecmax(int n, const double *v, unsigned long long *out, cudaStream_t s);
cudaError_t launch_to_f32_scaled(int n, int nrhs, const double *R, int ldr, const unsigned long long *rmax, float *R32,
                                 int ldr32, cudaStream_t s);
cudaError_t launch_axpy_scaled(int n, int nrhs, const float *D32, int ldd, const unsigned long long *rmax, double *X, int ldx,
                               cudaStream_t s);
// api.cu
int solve_f32_perm(int n, int nrhs, const float *LU, int lda, const int *perm, float *B, int ldb, cudaStream_t s,
                   const float *Dinv = nullptr);
int solve_f64_perm(int n, int nrhs, const double *LU, int lda, const int *perm, double *B, int ldb, cudaStream_t s,
                   const double *Dinv = nullptr);
size_t f32_diag_inverse_elems(int n);
size_t f64_diag_inverse_elems(int n);
int f32_diag_inverse(int n, const float *LU, int lda, float *Dinv, cudaStream_t s);
int f64_diag_inverse(int n, const double *LU, int lda, double *Dinv, cudaStream_t s);
int factor_f32_internal(int n, float *A, int lda, int *ipiv, int *info, int *perm, const lu_opts *o, cudaStream_t s);
int factor_f64_internal(int n, double *A, int lda, int *ipiv, int *info, int *perm, const lu_opts *o, cudaStream_t s);
CtaTrace cta_tag_ext(int kind, int step);   // the per-CTA trace argument of a launch
int default_outer_width(lu_dtype dt, int n, int update);   // the built-in b_o
// mixed.cu (continued)
cudaError_t launch_fill_probe(int n, unsigned long long seed, float *R32, cudaStream_t s);
cudaError_t launch_axpy_f64(int n, int nrhs, const double *D, int ldd, double *X, int ldx, cudaStream_t s);
cudaError_t launch_absmax_scaled_f32(int n, int nrhs, const float *D32, int ldd, const unsigned long long *rmax,
                                     unsigned long long *out, cudaStream_t s);
// gmres.cu
int gmres_ir(int n, int nrhs, const double *A, int lda, const double *B, int ldb, double *X, int ldx, const float *LU32,
             int ld32, const int *perm, double anorm, const double *bnorm, double tol, int max_outer, int restart,
             int *iters_out, int *inner_out, double *eta_out, cudaStream_t s, double budget_ms, const float *Dinv);
}  // namespace lu
