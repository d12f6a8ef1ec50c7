// stb_toeplitz.cu -- block-Toeplitz matrix-vector product (eq. V_mat):
//   y_r^k = beta y_r^k + sum_{d=0}^{k} A^d x_r^{k-d}
// FP64 arithmetic on the SIMT FP64 pipe.  The product is a sum of dense
// E x E by E x (n_steps - d) products, one per block d; the work is cut into
// items (64 rows of l) x (16 time columns k) x (8 blocks d) so that every SM
// gets a balanced share even though block d only feeds the columns k >= d.
// Each item accumulates into its own partial slice; a second kernel adds the
// slices in a fixed order (deterministic result).
#include <mutex>

#include "stb_internal.h"
#include "stb_toeplitz.h"
#include "stb_toeplitz_tc.h"

namespace stb {

constexpr int TM = 64;   // rows per item
constexpr int TK = 16;   // time columns per item
constexpr int TD = 8;    // blocks d per item
constexpr int TJ = 32;   // contraction chunk
constexpr int MV_THREADS = 128;

template <class AT>
__global__ void __launch_bounds__(MV_THREADS)
k_toeplitz_partial(const AT *__restrict__ A, int E, int n_steps, int nrhs,
                   const double *__restrict__ x, double *__restrict__ part) {
    __shared__ double As[TM][TJ + 1];
    __shared__ double Xs[TK][TJ + 1];
    const int n_kt = (n_steps + TK - 1) / TK;
    const int lt = blockIdx.x, kt = blockIdx.y % n_kt, r = blockIdx.y / n_kt, dr = blockIdx.z;
    const int l0 = lt * TM, k0 = kt * TK, d0 = dr * TD;
    if (d0 > k0 + TK - 1 || d0 >= n_steps) return;  // block range feeds no column here
    const int d1 = min(min(d0 + TD, n_steps), k0 + TK);
    const int tx = threadIdx.x % TK, ty = threadIdx.x / TK;  // column, row group (8 rows)
    double acc[TM / (MV_THREADS / TK)];
#pragma unroll
    for (int i = 0; i < TM / (MV_THREADS / TK); ++i) acc[i] = 0.0;
    const size_t EE = (size_t)E * E;
    const double *xr = x + (size_t)r * n_steps * E;
    for (int d = d0; d < d1; ++d) {
        const AT *Ad = A + (size_t)d * EE;
        for (int j0 = 0; j0 < E; j0 += TJ) {
            for (int t = threadIdx.x; t < TM * TJ; t += MV_THREADS) {
                int i = t / TJ, jj = t % TJ, l = l0 + i, j = j0 + jj;
                As[i][jj] = (l < E && j < E) ? (double)Ad[(size_t)l * E + j] : 0.0;
            }
            for (int t = threadIdx.x; t < TK * TJ; t += MV_THREADS) {
                int c = t / TJ, jj = t % TJ, k = k0 + c, j = j0 + jj;
                Xs[c][jj] = (k < n_steps && k - d >= 0 && j < E) ? xr[(size_t)(k - d) * E + j] : 0.0;
            }
            __syncthreads();
#pragma unroll 8
            for (int jj = 0; jj < TJ; ++jj) {
                double xv = Xs[tx][jj];
#pragma unroll
                for (int i = 0; i < TM / (MV_THREADS / TK); ++i)
                    acc[i] = fma(As[ty * (TM / (MV_THREADS / TK)) + i][jj], xv, acc[i]);
            }
            __syncthreads();
        }
    }
    const int k = k0 + tx;
    if (k >= n_steps) return;
    double *pr = part + (((size_t)dr * nrhs + r) * n_steps + k) * E;
#pragma unroll
    for (int i = 0; i < TM / (MV_THREADS / TK); ++i) {
        int l = l0 + ty * (TM / (MV_THREADS / TK)) + i;
        if (l < E) pr[l] = acc[i];
    }
}

// y = beta y + sum over the d-slices that feed column k (fixed order)
__global__ void k_toeplitz_reduce(const double *__restrict__ part, int E, int n_steps, int nrhs,
                                  double beta, double *__restrict__ y) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)nrhs * n_steps * E;
    if (idx >= total) return;
    int k = (int)((idx / E) % n_steps);
    size_t slice = total;
    double s = 0.0;
    for (int dr = 0; dr * TD <= k; ++dr) s += part[dr * slice + idx];
    y[idx] = beta == 0.0 ? s : fma(beta, y[idx], s);
}

size_t toeplitz_partial_bytes(int64_t E, int32_t n_steps, int32_t nrhs) {
    size_t n_dr = (n_steps + TD - 1) / TD;
    return align256(n_dr * (size_t)nrhs * n_steps * E * sizeof(double));
}

stb_status toeplitz_fp64(const void *A, int32_t storage, int64_t E, int32_t n_steps, int32_t nrhs,
                         const double *x, double beta, double *y, double *part, cudaStream_t s) {
    int n_kt = (n_steps + TK - 1) / TK, n_dr = (n_steps + TD - 1) / TD;
    dim3 grid((unsigned)((E + TM - 1) / TM), (unsigned)(n_kt * nrhs), (unsigned)n_dr);
    count_launch(s);
    if (storage == STB_STORE_F64)
        k_toeplitz_partial<double><<<grid, MV_THREADS, 0, s>>>((const double *)A, (int)E, n_steps,
                                                               nrhs, x, part);
    else
        k_toeplitz_partial<float><<<grid, MV_THREADS, 0, s>>>((const float *)A, (int)E, n_steps,
                                                              nrhs, x, part);
    stb_status st = check_launch("k_toeplitz_partial");
    if (st) return st;
    size_t total = (size_t)nrhs * n_steps * E;
    count_launch(s);
    k_toeplitz_reduce<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(part, (int)E, n_steps, nrhs,
                                                                      beta, y);
    return check_launch("k_toeplitz_reduce");
}

// ------------------------------------------------- double-float product ---
__global__ void k_split(const double *__restrict__ x, size_t n, float2 *__restrict__ xs) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    const float hi = (float)v;
    xs[i] = make_float2(hi, (float)(v - (double)hi));
}

// a (w_hi + w_lo) = p + e (p the FP32 product, e its error by FMA) plus the
// small w_lo term, accumulated into (hi, lo) by an error-free two-sum.
__device__ __forceinline__ void df_acc(float a, float2 x, float &hi, float &lo) {
    const float p = a * x.x;
    const float e = fmaf(a, x.x, -p);
    const float t = fmaf(a, x.y, e);
    const float s = hi + p;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += err + t;
}

__global__ void __launch_bounds__(MV_THREADS)
k_toeplitz_df_partial(const float *__restrict__ A, int E, int n_steps, int nrhs,
                      const float2 *__restrict__ xs, double *__restrict__ part) {
    __shared__ float As[TM][TJ + 1];
    __shared__ float2 Xs[TK][TJ + 1];
    const int n_kt = (n_steps + TK - 1) / TK;
    const int lt = blockIdx.x, kt = blockIdx.y % n_kt, r = blockIdx.y / n_kt, dr = blockIdx.z;
    const int l0 = lt * TM, k0 = kt * TK, d0 = dr * TD;
    if (d0 > k0 + TK - 1 || d0 >= n_steps) return;
    const int d1 = min(min(d0 + TD, n_steps), k0 + TK);
    const int tx = threadIdx.x % TK, ty = threadIdx.x / TK;
    constexpr int RPT = TM / (MV_THREADS / TK);  // rows per thread
    float hi[RPT], lo[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) hi[i] = lo[i] = 0.f;
    const size_t EE = (size_t)E * E;
    const float2 *xr = xs + (size_t)r * n_steps * E;
    for (int d = d0; d < d1; ++d) {
        const float *Ad = A + (size_t)d * EE;
        for (int j0 = 0; j0 < E; j0 += TJ) {
            for (int t = threadIdx.x; t < TM * TJ; t += MV_THREADS) {
                int i = t / TJ, jj = t % TJ, l = l0 + i, j = j0 + jj;
                As[i][jj] = (l < E && j < E) ? Ad[(size_t)l * E + j] : 0.f;
            }
            for (int t = threadIdx.x; t < TK * TJ; t += MV_THREADS) {
                int c = t / TJ, jj = t % TJ, k = k0 + c, j = j0 + jj;
                Xs[c][jj] = (k < n_steps && k - d >= 0 && j < E) ? xr[(size_t)(k - d) * E + j]
                                                                   : make_float2(0.f, 0.f);
            }
            __syncthreads();
#pragma unroll 4
            for (int jj = 0; jj < TJ; ++jj) {
                const float2 xv = Xs[tx][jj];
#pragma unroll
                for (int i = 0; i < RPT; ++i) df_acc(As[ty * RPT + i][jj], xv, hi[i], lo[i]);
            }
            __syncthreads();
        }
    }
    const int k = k0 + tx;
    if (k >= n_steps) return;
    double *pr = part + (((size_t)dr * nrhs + r) * n_steps + k) * E;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        int l = l0 + ty * RPT + i;
        if (l < E) pr[l] = (double)hi[i] + (double)lo[i];
    }
}

__global__ void k_toeplitz_df_reduce(const double *__restrict__ part, int E, int n_steps, int nrhs,
                                     int mode, const double *__restrict__ f, double beta,
                                     double *__restrict__ y) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)nrhs * n_steps * E;
    if (idx >= total) return;
    int k = (int)((idx / E) % n_steps);
    double s = 0.0;
    for (int dr = 0; dr * TD <= k; ++dr) s += part[dr * total + idx];
    if (mode == DF_RESIDUAL)
        y[idx] = f[idx] - s;
    else
        y[idx] = beta == 0.0 ? s : fma(beta, y[idx], s);
}

size_t toeplitz_df_bytes(int64_t E, int32_t n_steps, int32_t nrhs) {
    return toeplitz_partial_bytes(E, n_steps, nrhs) +
           align256((size_t)nrhs * n_steps * E * sizeof(float2));
}

stb_status toeplitz_df(const float *A, int64_t E, int32_t n_steps, int32_t nrhs, const double *x,
                       int mode, const double *f, double beta, double *y, void *scratch,
                       cudaStream_t s) {
    double *part = static_cast<double *>(scratch);
    float2 *xs = reinterpret_cast<float2 *>(static_cast<char *>(scratch) +
                                            toeplitz_partial_bytes(E, n_steps, nrhs));
    const size_t total = (size_t)nrhs * n_steps * E;
    count_launch(s);
    k_split<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(x, total, xs);
    stb_status st = check_launch("k_split");
    if (st) return st;
    int n_kt = (n_steps + TK - 1) / TK, n_dr = (n_steps + TD - 1) / TD;
    dim3 grid((unsigned)((E + TM - 1) / TM), (unsigned)(n_kt * nrhs), (unsigned)n_dr);
    count_launch(s);
    k_toeplitz_df_partial<<<grid, MV_THREADS, 0, s>>>(A, (int)E, n_steps, nrhs, xs, part);
    if ((st = check_launch("k_toeplitz_df_partial"))) return st;
    count_launch(s);
    k_toeplitz_df_reduce<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(part, (int)E, n_steps, nrhs,
                                                                         mode, f, beta, y);
    return check_launch("k_toeplitz_df_reduce");
}

// Scratch of stb_toeplitz_matvec_static: every device that loads the library
// holds these bytes until the process exits.  Host code must not hand the
// symbol itself to a kernel (on the host it names a host-side shadow); the
// device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_matvec_scratch[STB_TOEPLITZ_STATIC_SCRATCH_BYTES];

static stb_status matvec_scratch_address(double **out) {
    static std::mutex mu;
    static void *addr[256] = {};
    int dev = 0;
    STB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(STB_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_matvec_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(matvec scratch)");
        addr[dev] = p;
    }
    *out = static_cast<double *>(addr[dev]);
    return STB_OK;
}

}  // namespace stb

using namespace stb;

extern "C" stb_status stb_toeplitz_matvec_static(const void *A, int32_t a_storage, int64_t E,
                                                 int32_t n_steps, int32_t nrhs, const double *x,
                                                 double beta, double *y, stb_stream stream) {
    if (!A || !x || !y) return fail(STB_ERR_INVALID_ARG, "A, x and y must be given");
    if (a_storage != STB_STORE_F64 && a_storage != STB_STORE_F32)
        return fail(STB_ERR_INVALID_ARG, "a_storage must be STB_STORE_F64 or STB_STORE_F32");
    if (E < 1 || E > 65535 || n_steps < 1 || nrhs < 1)
        return fail(STB_ERR_INVALID_ARG, "need 1 <= E <= 65535, n_steps >= 1, nrhs >= 1");
    const size_t need = toeplitz_partial_bytes(E, n_steps, nrhs);
    if (need > STB_TOEPLITZ_STATIC_SCRATCH_BYTES)
        return fail(STB_ERR_INVALID_ARG,
                    "problem needs %zu bytes of scratch, the static scratch holds %zu; "
                    "use stb_toeplitz_matvec with a workspace",
                    need, (size_t)STB_TOEPLITZ_STATIC_SCRATCH_BYTES);
    double *part = nullptr;
    stb_status st = matvec_scratch_address(&part);
    if (st) return st;
    // every partial slice the reduction reads is written earlier in this call,
    // so the scratch needs no clearing
    return toeplitz_fp64(A, a_storage, E, n_steps, nrhs, x, beta, y, part, (cudaStream_t)stream);
}

extern "C" stb_status stb_toeplitz_workspace_size(int64_t E, int32_t n_steps, int32_t nrhs,
                                                  size_t *bytes) {
    if (!bytes || E < 1 || E > 65535 || n_steps < 1 || nrhs < 1)
        return fail(STB_ERR_INVALID_ARG, "need bytes, 1 <= E <= 65535, n_steps >= 1, nrhs >= 1");
    *bytes = 256 + toeplitz_partial_bytes(E, n_steps, nrhs);
    return STB_OK;
}

extern "C" stb_status stb_toeplitz_matvec(const void *A, int32_t a_storage, int64_t E,
                                          int32_t n_steps, int32_t nrhs, const double *x,
                                          double beta, double *y, void *ws, size_t ws_bytes,
                                          stb_stream stream) {
    if (!A || !x || !y) return fail(STB_ERR_INVALID_ARG, "A, x and y must be given");
    if (a_storage != STB_STORE_F64 && a_storage != STB_STORE_F32)
        return fail(STB_ERR_INVALID_ARG, "a_storage must be STB_STORE_F64 or STB_STORE_F32");
    size_t need;
    stb_status st = stb_toeplitz_workspace_size(E, n_steps, nrhs, &need);
    if (st) return st;
    if ((st = check_workspace(ws, ws_bytes, need))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    double *part = reinterpret_cast<double *>(static_cast<char *>(ws) + 256);
    return toeplitz_fp64(A, a_storage, E, n_steps, nrhs, x, beta, y, part, s);
}

extern "C" stb_status stb_toeplitz_ex_workspace_size(int64_t E, int32_t n_steps, int32_t nrhs,
                                                     int32_t arith, size_t *bytes) {
    stb_status st = stb_toeplitz_workspace_size(E, n_steps, nrhs, bytes);
    if (st) return st;
    switch (arith) {
    case STB_ARITH_FP64: return STB_OK;
    case STB_ARITH_DF: *bytes = 256 + toeplitz_df_bytes(E, n_steps, nrhs); return STB_OK;
    case STB_ARITH_TF32: *bytes = 256 + toeplitz_tc_bytes(E, n_steps, nrhs); return STB_OK;
    default: return fail(STB_ERR_INVALID_ARG, "arith must be STB_ARITH_FP64, _DF or _TF32");
    }
}

extern "C" stb_status stb_toeplitz_matvec_ex(const void *A, int32_t a_storage, int64_t E,
                                             int32_t n_steps, int32_t nrhs, const double *x,
                                             double beta, double *y, int32_t arith, void *ws,
                                             size_t ws_bytes, stb_stream stream) {
    if (arith == STB_ARITH_FP64)
        return stb_toeplitz_matvec(A, a_storage, E, n_steps, nrhs, x, beta, y, ws, ws_bytes, stream);
    if (!A || !x || !y) return fail(STB_ERR_INVALID_ARG, "A, x and y must be given");
    if (a_storage != STB_STORE_F32)
        return fail(STB_ERR_INVALID_ARG, "STB_ARITH_DF and STB_ARITH_TF32 need STB_STORE_F32 blocks");
    size_t need;
    stb_status st = stb_toeplitz_ex_workspace_size(E, n_steps, nrhs, arith, &need);
    if (st) return st;
    if ((st = check_workspace(ws, ws_bytes, need))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    void *scratch = static_cast<char *>(ws) + 256;
    if (arith == STB_ARITH_DF)
        return toeplitz_df((const float *)A, E, n_steps, nrhs, x, DF_AXPBY, nullptr, beta, y,
                           scratch, s);
    return toeplitz_tc((const float *)A, E, n_steps, nrhs, x, beta, y, scratch, status_word(ws), s);
}
