// stb_dense.h -- internal interface of the dense SPD helpers of the solve.
#pragma once
#include "stb_internal.h"

namespace stb {
// Scratch bytes of spd_inverse for an n x n matrix.
size_t spd_inverse_bytes(int64_t n);
// Inverse of the SPD FP64 matrix M (device, row-major n x n, unchanged):
// blocked Cholesky, inverse of the factor, M^{-1} = L^{-T} L^{-1}; *inv
// points into `scratch`.  A pivot that is not positive sets STB_ERR_NOT_SPD
// in *status (device).
stb_status spd_inverse(const double *M, int64_t n, void *scratch, size_t cap, int32_t *status,
                       double **inv, cudaStream_t s);
// out_v = A in_v, v = 0..nvec-1, vectors of length n contiguous (FP64).
stb_status dense_apply(const double *A, int64_t n, int64_t nvec, const double *in, double *out,
                       cudaStream_t s);
}  // namespace stb
