// stb_toeplitz_tc.h -- internal interface of the tensor-core (tcgen05, TF32)
// block-Toeplitz product.
#pragma once
#include "stb_internal.h"

namespace stb {
// Scratch bytes of toeplitz_tc (padded FP32 copy of x and partial sums).
size_t toeplitz_tc_bytes(int64_t E, int32_t n_steps, int32_t nrhs);
// y = beta y + T(A) x with FP32 blocks A read as TF32 by the tensor cores, x
// rounded to TF32, FP32 accumulation per slice of blocks and an FP64 sum of
// the slices.  Needs E % 4 == 0 and A 16-byte aligned.  A bounded wait that
// expires writes STB_ERR_TIMEOUT to *status (device).
stb_status toeplitz_tc(const float *A, int64_t E, int32_t n_steps, int32_t nrhs, const double *x,
                       double beta, double *y, void *scratch, int32_t *status, cudaStream_t s);
}  // namespace stb
