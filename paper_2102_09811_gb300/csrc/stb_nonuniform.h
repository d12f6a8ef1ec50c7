// stb_nonuniform.h -- internal interface of the non-uniform time grid products.
#pragma once
#include "stb_internal.h"

namespace stb {
// y^k = sum_{i <= k} A^{k,i} x^i, blocks packed at k(k+1)/2 + i (FP64).
stb_status matvec_nu(const double *A, int64_t E, int n_steps, int nrhs, const double *x,
                     double *y, cudaStream_t s);
}  // namespace stb
