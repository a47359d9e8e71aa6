// Internal host-side launchers and kernel pointers (not part of the public C ABI).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

namespace podcg {

struct DevState;
struct ProbDesc;

int grid_rows(int rows, int per_block, int sms);
void set_last_error(const std::string& msg);   // message for pod_cg_last_error(NULL)
int spmv_lanes_for(double mean_row);
int wb_bucket(int w);

// sparse
cudaError_t launch_spmv_plain(int L, const int32_t* rp, const int32_t* col, const double* val, const double* x,
                              double* y, int n, int sms, cudaStream_t s);
cudaError_t launch_spmv_plain32(int L, const int32_t* rp, const int32_t* col, const float* val, const float* x,
                                float* y, int n, int sms, cudaStream_t s);
void* kernel_spmv_cg(int L, bool fp32);
void* kernel_residual(int L, bool cond);
cudaError_t launch_spmm(const int32_t* rp, const int32_t* col, const double* val, const double* W, int ldw,
                        double* AW, int lda, int n, int w, int sms, cudaStream_t s);
cudaError_t launch_spmm_f32(const int32_t* rp, const int32_t* col, const float* val, const float* W, int ldw,
                            float* AW, int lda, int n, int w, int sms, cudaStream_t s);
cudaError_t launch_dinv(const ProbDesc* pd, int n, double* dinv, float* dinv32, DevState* st, int sms,
                        cudaStream_t s);
cudaError_t launch_to_f32(const double* a, float* b, size_t m, int sms, cudaStream_t s);
cudaError_t launch_desc_val_to_f32(const ProbDesc* pd, float* v32, int64_t nnz, int sms, cudaStream_t s);

// 3x3 block-sparse form of the CG product (k_bsr.cu)
cudaError_t launch_bsr_check(const int32_t* rp, const int32_t* col, int n, int* bad, int sms, cudaStream_t s);
cudaError_t launch_bsr_pattern(const int32_t* rp, const int32_t* col, int nb, int32_t* brp, int32_t* bcol, int sms,
                               cudaStream_t s);
cudaError_t launch_bsr_values(const int32_t* rp, const double* val, int n, int nnzb, double* bval, float* bval32,
                              int sms, cudaStream_t s);
int bsr_lanes_for(double blocks_per_row);
void* kernel_bsr_spmv_cg(int L, bool fp32);

// dense
void gram_shape(int n, int p, int q, int sms, int* tiles_j, int* tiles, int* splits, int* rows_per_split);
size_t gram_workspace_bytes(int n, int p, int q, int sms);
cudaError_t launch_gram_reduce(const double* work, int splits, int tiles, int tj, int p, int q, double* G, int ldg,
                               cudaStream_t s);
cudaError_t launch_gram(int n, const double* X, int ldx, int p, const double* Y, int ldy, int qy,
                        const double* extra, double* G, int ldg, int upper_only, double* work,
                        size_t work_bytes, int sms, cudaStream_t s);
cudaError_t launch_lift(int n, const double* S, int lds, int s, const double* C, const DevState* st,
                        double* W, int ldw, int sms, cudaStream_t str, int cols_y = 0);
cudaError_t launch_stage1(int wb, const ProbDesc* pd, int n, const double* W, const double* AW, double* x,
                          double* r, double* partials, unsigned int* counter, DevState* st, double tol, int sms,
                          cudaStream_t s);
cudaError_t launch_pod_eig(const double* G, int ldg, int s, double energy, double rank_tol, int w_max, double* C,
                           double* sigma2, DevState* st, double* Vprev, int prev_s, cudaStream_t str,
                           double energy_y = 1.0, int y_max = 0);
// M = R^{-1} R^{-T} of the current basis (st->w), row stride kWMax (k_dense.cu)
cudaError_t launch_mu_matrix(const double* Rinv, const DevState* st, double* M, cudaStream_t str);
cudaError_t launch_chol(const double* G, int ldg, double* Rinv, DevState* st, int want_cond, cudaStream_t str,
                        int w_dim = -1, int truncate = 0);
cudaError_t launch_gram_scatter(const double* row, int s, int q, double* G, int ldg, cudaStream_t str);
cudaError_t launch_cs_gram(const double* cs, int ldc, int s, int q, double* G, int ldg, cudaStream_t str);
cudaError_t launch_symmetrize(double* G, int ldg, int s, cudaStream_t str);
// accumulated Krylov vectors (k_dense.cu): previous / RBF weights and column scaling
cudaError_t launch_krylov_coords(const double* G, int ldg, int z, double rcond, double* coords, double* eta, int rbf,
                                 cudaStream_t str);
cudaError_t launch_scale_cols(const double* src, double* dst, int ld, int n, int k, const double* f, int inv_sqrt,
                              int sms, cudaStream_t str);

// CG iteration (k_cg.cu): kernel pointers for graph construction
// FP32 with w > 0 has two forms of the update/direction passes: row-parallel float4
// (kProjDirect) and tiles staged by the TMA engine (kProjStaged: one CTA of
// tma_block_threads() threads per SM, tma_grid() CTAs, dynamic shared memory returned in
// bytes, the panels passed as tensor maps; 0 for every other kernel). w16: the staged
// direction pass reads the 16-bit copy of W (with its column scales).
constexpr int kProjDirect = 0;
constexpr int kProjStaged = 1;
void cg_kernels(int wb, bool fp32, bool cond, int form, bool w16, void** init, void** upd, void** dir0, void** dir,
                int* smem_upd, int* smem_dir);
int tma_block_threads();
// launch shape of a TMA-staged pass over ncols panel columns (cols_per_box per box: 8 FP32,
// 16 fp16) and nvec vector tiles per stage (two CTAs per SM when allow_pair and the stage is
// small): grid, ring bytes (a kernel argument) and the dynamic shared memory
void tma_shape(int n, int sms, int ncols, int cols_per_box, int nvec, bool allow_pair, int* grid, int* ring_bytes,
               int* smem);
// W16 = the 16-bit copy of the FP32 basis W32 with power-of-two column scales, and W32
// replaced by its exact dequantised value (k_cg.cu); cmax: kWMax words of scratch
cudaError_t launch_quant16(int n, int ld, float* W32, __half* W16, unsigned int* cmax, float* wscale,
                           const DevState* st, int sms, cudaStream_t s);
// a 2D tensor map over a column-major panel (rows = ld, cols columns, element 2, 4 or 8
// bytes) with boxes of 256 rows x box_cols columns, no swizzle, zero fill past the rows
bool encode_panel_map(CUtensorMap* tm, const void* base, int elem_bytes, int ld, int cols, int box_cols);

// stage two of the three-stage algorithm (k_stage2.cu, FP64): kernel pointers for graph
// construction, y = the augmenting-basis dimension (selects the width bucket), L = SpMV lanes
void stage2_kernels(int y, int L, bool cond, void** bb, void** init, void** lift, void** apply);
// stage three over the entire augmenting basis (k_stage2.cu, FP64): the augmentation step
// A z -> Y^T A z with the inner solve's start, the first and later direction updates with Y,
// and the switch of the update kernels to no basis
void it_kernels(int y, int L, void** az, void** dir0, void** dir, void** begin);
cudaError_t launch_s2_to_f32(int n, int ld, const double* W, float* W32, int col0, int ncols, const double* Rinv,
                             int sms, cudaStream_t s);

// mixed precision (k_mixed.cu)
void mixed_kernels(int wb, void** proj, void** start);
void* kernel_mx_accum();
cudaError_t launch_lift32(int n, const float* S, int lds, int s, const double* C, const DevState* st, float* W,
                          int ldw, int sms, cudaStream_t str, int cols_y = 0);
cudaError_t launch_stage1_mx(int wb, const ProbDesc* pd, int n, const float* W32, double* x, double* partials,
                             unsigned int* counter, DevState* st, double tol, int sms, cudaStream_t s);
cudaError_t launch_gram32(int n, const float* X, int ldx, int p, const float* Y, int ldy, int qy, const double* extra,
                          double* G, int ldg, int upper_only, double* work, size_t work_bytes, int sms,
                          cudaStream_t s);

// the wait override of pod_cg_debug_wait_timeout for the current device, per unit
cudaError_t gram_tc_set_wait_test(int mask, long long cycles);
cudaError_t cg_set_wait_test(int mask, long long cycles);
cudaError_t loop_set_wait_test(int mask, long long cycles);

// the FP32 inner loop as one persistent cooperative kernel (k_loop.cu): kernel pointer for a
// basis-width bucket (0 or 8; NULL otherwise) and its grid (every CTA resident; 0 = none)
void* kernel_cg_loop(int wb);
int cg_loop_grid(int wb, int sms);

// tensor-core Gram with split-bf16 products (k_gram_tc.cu); G = X^T [Y, extra]
size_t gram_tc_workspace_bytes(int n, int p, int q, int sms);
bool gram_tc_aligned(const void* ptr, size_t ld_bytes);
cudaError_t launch_gram_tc(int n, const float* X, int ldx, int p, const float* Y, int ldy, int qy,
                           const double* extra, double* G, int ldg, double* work, size_t work_bytes, int* err_flag,
                           int sms, cudaStream_t s);
cudaError_t launch_gram_tc(int n, const double* X, int ldx, int p, const double* Y, int ldy, int qy,
                           const double* extra, double* G, int ldg, double* work, size_t work_bytes, int* err_flag,
                           int sms, cudaStream_t s);

// differentiation (k_adjoint.cu)
cudaError_t launch_diffusion_assemble(int mx, int my, int mz, const double* theta, const double* extra,
                                      const int32_t* rp, double* val, int sms, cudaStream_t s);
cudaError_t launch_theta_grad(int mx, int my, int mz, const double* theta, int nsys, const double* lam,
                              const double* xs, double* grad, int sms, cudaStream_t s);

// batched persistent solver (k_batch.cu)
struct BatchSeqDev;
int batch_max_clusters(int cluster);
size_t batch_smem_bytes();
cudaError_t launch_batch(const BatchSeqDev* seqs, const int* order, int nseq, unsigned int* ticket, int cluster,
                         int grid_clusters, int k_max, int max_refine, double inner_tol, double rank_tol,
                         cudaStream_t s);

}  // namespace podcg
