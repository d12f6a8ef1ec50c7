// stb_toeplitz.h -- internal interface of the block-Toeplitz product.
#pragma once
#include "stb_internal.h"

namespace stb {
size_t toeplitz_partial_bytes(int64_t E, int32_t n_steps, int32_t nrhs);
// y = beta y + T(A) x in FP64; `part` has toeplitz_partial_bytes() bytes.
stb_status toeplitz_fp64(const void *A, int32_t storage, int64_t E, int32_t n_steps, int32_t nrhs,
                         const double *x, double beta, double *y, double *part, cudaStream_t s);
// The blockwise transpose: y^k = beta y^k + sum_d (A^d)^T x^{k-d} with A^d
// stored [E][N], x [nrhs][n_steps][E], y [nrhs][n_steps][N]; `part` has
// toeplitz_partial_bytes(N, ...) bytes.
stb_status toeplitz_fp64_rect_t(const void *A, int32_t storage, int64_t E, int64_t N,
                                int32_t n_steps, int32_t nrhs, const double *x, double beta,
                                double *y, double *part, cudaStream_t s);
// The same with rectangular blocks A^d [E][N]: x [nrhs][n_steps][N],
// y [nrhs][n_steps][E]; `part` has toeplitz_partial_bytes(E, ...) bytes.
stb_status toeplitz_fp64_rect(const void *A, int32_t storage, int64_t E, int64_t N, int32_t n_steps,
                              int32_t nrhs, const double *x, double beta, double *y, double *part,
                              cudaStream_t s);

// The same product for FP32 blocks in FP32-pair ("double-float") arithmetic:
// exact FP32 products with a two-float split of x, error-free two-sums, so
// the result carries about 44 significant bits without FP64 instructions.
//   mode DF_AXPBY:    y = beta y + T(A) x
//   mode DF_RESIDUAL: y = f - T(A) x
enum { DF_AXPBY = 0, DF_RESIDUAL = 1 };
size_t toeplitz_df_bytes(int64_t E, int32_t n_steps, int32_t nrhs);
stb_status toeplitz_df(const float *A, int64_t E, int32_t n_steps, int32_t nrhs, const double *x,
                       int mode, const double *f, double beta, double *y, void *scratch,
                       cudaStream_t s);
// The same with an FP32 vector x (exactly representable: no low part);
// f may alias y in mode DF_RESIDUAL.
stb_status toeplitz_df_f32x(const float *A, int64_t E, int32_t n_steps, int32_t nrhs,
                            const float *x, int mode, const double *f, double beta, double *y,
                            void *scratch, cudaStream_t s);
// y = A x (overwritten) for FP32 blocks of E rows and N columns, FP64 x of
// length N and y of length E per step, in the same double-float arithmetic;
// scratch of toeplitz_df_rect_bytes.
size_t toeplitz_df_rect_bytes(int64_t E, int64_t N, int32_t n_steps, int32_t nrhs);
stb_status toeplitz_df_rect(const float *A, int64_t E, int64_t N, int32_t n_steps, int32_t nrhs,
                            const double *x, double *y, void *scratch, cudaStream_t s);

// The same product on the tcgen05 tensor cores with split operands (bf16
// digit slices, exact FP32 accumulation per 64-column chunk, double-float
// sums across chunks): error about 2^-44 of the chunk magnitudes.  Any E;
// scratch of toeplitz_split_bytes; a bounded wait that expires writes
// STB_ERR_TIMEOUT to *status (device).  Block entries must lie below 2^126 in
// magnitude.  f may alias y in mode DF_RESIDUAL.  a_exp_ready: the scratch
// already holds A's row exponents from an earlier call with the same A and
// sizes (the refinement residuals of one solve), so the pass over A that
// forms them is skipped.
size_t toeplitz_split_bytes(int64_t E, int32_t n_steps, int32_t nrhs);
stb_status toeplitz_split(const float *A, int64_t E, int32_t n_steps, int32_t nrhs, const double *x,
                          int mode, const double *f, double beta, double *y, void *scratch,
                          int32_t *status, cudaStream_t s);
stb_status toeplitz_split_f32x(const float *A, int64_t E, int32_t n_steps, int32_t nrhs,
                               const float *x, int mode, const double *f, double beta, double *y,
                               void *scratch, int32_t *status, bool a_exp_ready, cudaStream_t s);

// Far history of a panel of 8 steps of the march on the tensor cores (three
// floating bf16 slices per operand, six products, FP32 accumulation; FP32
// accuracy), for FP32 blocks V and the FP32 march vector x [nrhs][n_steps][E]
// of up to 8 right-hand sides:
//   part[z][r][c][l] = sum over the blocks of slice z of V^d[l,:] x_r^{kp+c-d}
// restricted to 0 <= kp + c - d < kp (c < nb <= 8), z < *n_z (at most
// panel_tc_max_slices()).
// `xf` (panel_tc_bytes) holds the slices of the solved steps: clear it with
// panel_tc_begin before the first panel of a march; each call slices the
// steps kp-8 .. kp-1 (panels in order).
bool panel_tc_supported(int32_t nrhs);
bool panel_tc_blocks_ok(const float *V, int64_t E);
size_t panel_tc_bytes(int64_t E, int32_t n_steps, int32_t nrhs);
int panel_tc_max_slices();
stb_status panel_tc_begin(int64_t E, int32_t n_steps, int32_t nrhs, void *xf, cudaStream_t s);
stb_status panel_tc(const float *V, int64_t E, int32_t n_steps, int32_t nrhs, const float *x,
                    int kp, int nb, void *xf, float *part, int *n_z, int32_t *status,
                    cudaStream_t s);
}  // namespace stb
