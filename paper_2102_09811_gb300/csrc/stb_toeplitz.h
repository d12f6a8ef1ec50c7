// stb_toeplitz.h -- internal interface of the block-Toeplitz product.
#pragma once
#include "stb_internal.h"

namespace stb {
size_t toeplitz_partial_bytes(int64_t E, int32_t n_steps, int32_t nrhs);
// y = beta y + T(A) x in FP64; `part` has toeplitz_partial_bytes() bytes.
stb_status toeplitz_fp64(const void *A, int32_t storage, int64_t E, int32_t n_steps, int32_t nrhs,
                         const double *x, double beta, double *y, double *part, cudaStream_t s);
}  // namespace stb
