// stb_nonuniform.cu -- block lower-triangular products and the block
// forward substitution on a non-uniform time grid (Sec. 7: the temporal
// antiderivatives carry over, the matrices lose their Toeplitz structure).
// Blocks A^{k,i} (k >= i) are packed at b(k,i) = k(k+1)/2 + i, each E x E
// row-major FP64; vectors are [nrhs][n_steps][E].  FP64 throughout.
#include <algorithm>

#include "stb_dense.h"
#include "stb_internal.h"
#include "stb_nonuniform.h"

namespace stb {

constexpr int NU_THREADS = 256;

// out_{r,k}[l] = base_{r,k}[l] + sign sum_{i < imax} sum_j A^{k,i}[l][j] x_{r,i}[j]
// for one step k (imax = k + 1: the whole block row; imax = k: the history),
// one warp per (r, l); base may be null.
__global__ void __launch_bounds__(NU_THREADS)
k_blockrow_nu(const double *__restrict__ A, int E, int n_steps, int nrhs, int k, int imax,
              const double *__restrict__ x, const double *__restrict__ base, double sign,
              double *__restrict__ out, size_t out_stride) {
    const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= nrhs * E) return;
    const int r = warp / E, l = warp % E;
    double acc = 0.0;
    for (int i = 0; i < imax; ++i) {
        const double *row = A + (((size_t)k * (k + 1) / 2 + i) * E + l) * E;
        const double *xv = x + ((size_t)r * n_steps + i) * E;
        for (int j = lane; j < E; j += 32) acc = fma(row[j], xv[j], acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        const double b = base ? base[((size_t)r * n_steps + k) * E + l] : 0.0;
        out[(size_t)r * out_stride + l] = fma(sign, acc, b);
    }
}

// w_{r,k} = tmp_r (the solve's result for step k)
__global__ void k_put_step(const double *__restrict__ tmp, int E, int n_steps, int nrhs, int k,
                           double *__restrict__ w) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)nrhs * E) return;
    const int r = (int)(idx / E), l = (int)(idx % E);
    w[((size_t)r * n_steps + k) * E + l] = tmp[idx];
}

stb_status matvec_nu(const double *A, int64_t E, int n_steps, int nrhs, const double *x,
                     double *y, cudaStream_t s) {
    const unsigned blocks = (unsigned)(((size_t)nrhs * E * 32 + NU_THREADS - 1) / NU_THREADS);
    for (int k = 0; k < n_steps; ++k) {
        count_launch(s);
        k_blockrow_nu<<<blocks, NU_THREADS, 0, s>>>(A, (int)E, n_steps, nrhs, k, k + 1, x, nullptr,
                                                    1.0, y + (size_t)k * E, (size_t)n_steps * E);
        stb_status st = check_launch("k_blockrow_nu");
        if (st) return st;
    }
    return STB_OK;
}

struct NuSolveLayout {
    double *inv;   // [n_steps][E][E]: inverses of the diagonal blocks
    void *spd;     // scratch of spd_inverse
    size_t spd_bytes;
    double *t0, *t1;  // [nrhs][E]
    size_t bytes;
};

static NuSolveLayout nu_solve_layout(int64_t E, int n_steps, int nrhs, void *ws, size_t cap) {
    Carve c(ws, cap);
    NuSolveLayout L{};
    L.inv = c.take<double>((size_t)n_steps * E * E);
    L.spd_bytes = spd_inverse_bytes(E);
    L.spd = c.take<char>(L.spd_bytes);
    L.t0 = c.take<double>((size_t)nrhs * E);
    L.t1 = c.take<double>((size_t)nrhs * E);
    L.bytes = c.off;
    return L;
}

}  // namespace stb

using namespace stb;

extern "C" stb_status stb_matvec_nu(const double *A, int64_t E, int32_t n_steps, int32_t nrhs,
                                    const double *x, double *y, stb_stream stream) {
    if (!A || !x || !y || E < 1 || E > 65535 || n_steps < 1 || nrhs < 1)
        return fail(STB_ERR_INVALID_ARG, "invalid argument");
    return matvec_nu(A, E, n_steps, nrhs, x, y, (cudaStream_t)stream);
}

extern "C" stb_status stb_solve_nu_workspace_size(int64_t E, int32_t n_steps, int32_t nrhs,
                                                  size_t *bytes) {
    if (!bytes || E < 1 || E > 65535 || n_steps < 1 || nrhs < 1)
        return fail(STB_ERR_INVALID_ARG, "invalid argument");
    *bytes = align256(nu_solve_layout(E, n_steps, nrhs, nullptr, 0).bytes);
    return STB_OK;
}

extern "C" stb_status stb_solve_nu(const double *V, int64_t E, int32_t n_steps, int32_t nrhs,
                                   const double *f, double *w, void *ws, size_t ws_bytes,
                                   stb_stream stream) {
    if (!V || !f || !w) return fail(STB_ERR_INVALID_ARG, "null argument");
    size_t need;
    stb_status st = stb_solve_nu_workspace_size(E, n_steps, nrhs, &need);
    if (st) return st;
    if ((st = check_workspace(ws, ws_bytes, need))) return st;
    NuSolveLayout L = nu_solve_layout(E, n_steps, nrhs, ws, ws_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    int32_t *status = status_word(ws);
    const size_t EE = (size_t)E * E;
    for (int k = 0; k < n_steps; ++k) {  // every diagonal block has its own step length
        double *inv = nullptr;
        if ((st = spd_inverse(V + ((size_t)k * (k + 1) / 2 + k) * EE, E, L.spd, L.spd_bytes, status,
                              &inv, s)))
            return st;
        STB_CUDA(cudaMemcpyAsync(L.inv + (size_t)k * EE, inv, sizeof(double) * EE,
                                 cudaMemcpyDeviceToDevice, s));
    }
    const unsigned rows = (unsigned)(((size_t)nrhs * E * 32 + NU_THREADS - 1) / NU_THREADS);
    const unsigned put = (unsigned)(((size_t)nrhs * E + 255) / 256);
    for (int k = 0; k < n_steps; ++k) {
        // t0 = f^k - sum_{i<k} V^{k,i} w^i, then w^k = (V^{k,k})^{-1} t0
        count_launch(s);
        k_blockrow_nu<<<rows, NU_THREADS, 0, s>>>(V, (int)E, n_steps, nrhs, k, k, w, f, -1.0, L.t0,
                                                  (size_t)E);
        if ((st = check_launch("k_blockrow_nu"))) return st;
        if ((st = dense_apply(L.inv + (size_t)k * EE, E, nrhs, L.t0, L.t1, s))) return st;
        count_launch(s);
        k_put_step<<<put, 256, 0, s>>>(L.t1, (int)E, n_steps, nrhs, k, w);
        if ((st = check_launch("k_put_step"))) return st;
    }
    return stb_workspace_status(ws, stream);
}
