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

// TRANS: every block is stored transposed, as As^d [N][E] with
// A^d[l][j] = As^d[j][l] (the blockwise transpose of Sec. 3.2's remark).
template <class AT, bool TRANS = false>
__global__ void __launch_bounds__(MV_THREADS)
k_toeplitz_partial(const AT *__restrict__ A, int E, int N, int n_steps, int nrhs,
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
    const size_t EN = (size_t)E * N;
    const double *xr = x + (size_t)r * n_steps * N;
    for (int d = d0; d < d1; ++d) {
        const AT *Ad = A + (size_t)d * EN;
        for (int j0 = 0; j0 < N; j0 += TJ) {
            if (TRANS) {  // stored [N][E]: consecutive threads read consecutive l
                for (int t = threadIdx.x; t < TM * TJ; t += MV_THREADS) {
                    int jj = t / TM, i = t % TM, l = l0 + i, j = j0 + jj;
                    As[i][jj] = (l < E && j < N) ? (double)Ad[(size_t)j * E + l] : 0.0;
                }
            } else {
                for (int t = threadIdx.x; t < TM * TJ; t += MV_THREADS) {
                    int i = t / TJ, jj = t % TJ, l = l0 + i, j = j0 + jj;
                    As[i][jj] = (l < E && j < N) ? (double)Ad[(size_t)l * N + j] : 0.0;
                }
            }
            for (int t = threadIdx.x; t < TK * TJ; t += MV_THREADS) {
                int c = t / TJ, jj = t % TJ, k = k0 + c, j = j0 + jj;
                Xs[c][jj] = (k < n_steps && k - d >= 0 && j < N) ? xr[(size_t)(k - d) * N + j] : 0.0;
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
    return toeplitz_fp64_rect(A, storage, E, E, n_steps, nrhs, x, beta, y, part, s);
}

template <bool TRANS>
static stb_status toeplitz_rect_run(const void *A, int32_t storage, int64_t E, int64_t N,
                                    int32_t n_steps, int32_t nrhs, const double *x, double beta,
                                    double *y, double *part, cudaStream_t s) {
    int n_kt = (n_steps + TK - 1) / TK, n_dr = (n_steps + TD - 1) / TD;
    dim3 grid((unsigned)((E + TM - 1) / TM), (unsigned)(n_kt * nrhs), (unsigned)n_dr);
    count_launch(s);
    if (storage == STB_STORE_F64)
        k_toeplitz_partial<double, TRANS><<<grid, MV_THREADS, 0, s>>>(
            (const double *)A, (int)E, (int)N, n_steps, nrhs, x, part);
    else
        k_toeplitz_partial<float, TRANS><<<grid, MV_THREADS, 0, s>>>(
            (const float *)A, (int)E, (int)N, n_steps, nrhs, x, part);
    stb_status st = check_launch("k_toeplitz_partial");
    if (st) return st;
    size_t total = (size_t)nrhs * n_steps * E;
    count_launch(s);
    k_toeplitz_reduce<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(part, (int)E, n_steps, nrhs,
                                                                      beta, y);
    return check_launch("k_toeplitz_reduce");
}

stb_status toeplitz_fp64_rect_t(const void *A, int32_t storage, int64_t E, int64_t N,
                                int32_t n_steps, int32_t nrhs, const double *x, double beta,
                                double *y, double *part, cudaStream_t s) {
    return toeplitz_rect_run<true>(A, storage, N, E, n_steps, nrhs, x, beta, y, part, s);
}

stb_status toeplitz_fp64_rect(const void *A, int32_t storage, int64_t E, int64_t N, int32_t n_steps,
                              int32_t nrhs, const double *x, double beta, double *y, double *part,
                              cudaStream_t s) {
    int n_kt = (n_steps + TK - 1) / TK, n_dr = (n_steps + TD - 1) / TD;
    dim3 grid((unsigned)((E + TM - 1) / TM), (unsigned)(n_kt * nrhs), (unsigned)n_dr);
    count_launch(s);
    if (storage == STB_STORE_F64)
        k_toeplitz_partial<double><<<grid, MV_THREADS, 0, s>>>((const double *)A, (int)E, (int)N,
                                                               n_steps, nrhs, x, part);
    else
        k_toeplitz_partial<float><<<grid, MV_THREADS, 0, s>>>((const float *)A, (int)E, (int)N,
                                                              n_steps, nrhs, x, part);
    stb_status st = check_launch("k_toeplitz_partial");
    if (st) return st;
    size_t total = (size_t)nrhs * n_steps * E;
    count_launch(s);
    k_toeplitz_reduce<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(part, (int)E, n_steps, nrhs,
                                                                      beta, y);
    return check_launch("k_toeplitz_reduce");
}

// ------------------------------------------------- double-float product ---
// Blocks d per item: half of TD, so that a 64-step product over 3072 rows
// runs about 2.5 waves of resident CTAs instead of 1.3.
constexpr int DF_TD = 4;

static size_t df_partial_bytes(int64_t E, int32_t n_steps, int32_t nrhs) {
    const size_t n_dr = (n_steps + DF_TD - 1) / DF_TD;
    return align256(n_dr * (size_t)nrhs * n_steps * E * sizeof(double));
}
__global__ void k_split(const double *__restrict__ x, size_t n, float2 *__restrict__ xs) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    const float hi = (float)v;
    xs[i] = make_float2(hi, (float)(v - (double)hi));
}

// Two rows at once in packed FP32x2 arithmetic: a (w_hi + w_lo) = p + e
// (p the FP32 product, e its error by FMA) plus the small w_lo term,
// accumulated into (hi, lo) by an error-free two-sum.  Differences are
// written as u - v = fma(v, -1, u) (exact negation, one rounding) and the
// product is formed negated, pn = -p, so that no separate negation is needed.
__device__ __forceinline__ float2 sub2(float2 u, float2 v) {
    return __ffma2_rn(v, make_float2(-1.f, -1.f), u);
}
template <bool SPLIT>
__device__ __forceinline__ void df_acc2(float2 a, float2 xh, float2 nxh, float2 xl, float2 &hi,
                                        float2 &lo) {
    const float2 pn = __fmul2_rn(a, nxh);       // -p
    const float2 e = __ffma2_rn(a, xh, pn);      // a xh - p, exact
    const float2 t = SPLIT ? __ffma2_rn(a, xl, e) : e;  // x single-float: no low part
    const float2 s = sub2(hi, pn);               // hi + p
    const float2 bb = sub2(s, hi);
    const float2 c2 = sub2(hi, sub2(s, bb));     // hi - (s - bb)
    const float2 c3n = __fadd2_rn(pn, bb);       // -(p - bb)
    const float2 err = sub2(c2, c3n);
    hi = s;
    lo = __fadd2_rn(lo, __fadd2_rn(err, t));
}

// Item (64 rows l, 16 columns k, 8 blocks d) of the double-float product.
// A thread owns one column and 8 rows (4 packed pairs); the A tile is stored
// transposed in shared memory so that a pair of rows is one 8-byte word, and
// x as (hi, hi, lo, lo) so that both operands of the packed ops load as is.
// The (d, j) tiles are visited in one flat sequence and the next tile is
// loaded into registers while the current one is being multiplied.  VEC:
// E % 4 == 0 and A 16-byte aligned (rows loaded as float4).  SPLIT: x is a
// two-float split xs of an FP64 vector; otherwise x is the FP32 vector xf.
template <bool VEC, bool SPLIT>
__global__ void __launch_bounds__(MV_THREADS)
k_toeplitz_df_partial(const float *__restrict__ A, int E, int N, int n_steps, int nrhs,
                      const float2 *__restrict__ xs, const float *__restrict__ xf,
                      double *__restrict__ part) {
    __shared__ __align__(16) float As[TJ][TM + 4];
    __shared__ __align__(16) float4 Xs[TJ][TK];
    const int n_kt = (n_steps + TK - 1) / TK;
    const int lt = blockIdx.x, kt = blockIdx.y % n_kt, r = blockIdx.y / n_kt, dr = blockIdx.z;
    const int l0 = lt * TM, k0 = kt * TK, d0 = dr * DF_TD;
    if (d0 > k0 + TK - 1 || d0 >= n_steps) return;
    const int d1 = min(min(d0 + DF_TD, n_steps), k0 + TK);
    const int tx = threadIdx.x % TK, ty = threadIdx.x / TK;
    constexpr int RPT = TM / (MV_THREADS / TK);  // rows per thread (8)
    constexpr int AV = TM * TJ / 4 / MV_THREADS;  // float4 of the A tile per thread (4)
    constexpr int XV = TK * TJ / MV_THREADS;      // x values of the tile per thread (4)
    float2 hi[RPT / 2], lo[RPT / 2];
#pragma unroll
    for (int i = 0; i < RPT / 2; ++i) hi[i] = lo[i] = make_float2(0.f, 0.f);
    const size_t EE = (size_t)E * N;
    const float2 *xr = SPLIT ? xs + (size_t)r * n_steps * N : nullptr;
    const float *xfr = SPLIT ? nullptr : xf + (size_t)r * n_steps * N;
    const int n_j = (N + TJ - 1) / TJ, n_it = (d1 - d0) * n_j;

    float4 ra[AV];
    float2 rx[XV];
    auto load_tile = [&](int it) {
        const int d = d0 + it / n_j, j0 = (it % n_j) * TJ;
        const float *Ad = A + (size_t)d * EE;
#pragma unroll
        for (int v = 0; v < AV; ++v) {
            const int t = threadIdx.x + v * MV_THREADS;
            const int i = t / (TJ / 4), j = j0 + 4 * (t % (TJ / 4)), l = l0 + i;
            if (VEC) {
                ra[v] = (l < E && j < N) ? __ldg(reinterpret_cast<const float4 *>(Ad + (size_t)l * N + j))
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                const float *row = Ad + (size_t)l * N;
                const bool ok = l < E;
                ra[v] = make_float4(ok && j < N ? row[j] : 0.f, ok && j + 1 < N ? row[j + 1] : 0.f,
                                    ok && j + 2 < N ? row[j + 2] : 0.f,
                                    ok && j + 3 < N ? row[j + 3] : 0.f);
            }
        }
#pragma unroll
        for (int v = 0; v < XV; ++v) {
            const int t = threadIdx.x + v * MV_THREADS;
            const int jj = t / TK, c = t % TK, k = k0 + c, j = j0 + jj;
            const bool in = k < n_steps && k - d >= 0 && j < N;
            if (SPLIT)
                rx[v] = in ? xr[(size_t)(k - d) * N + j] : make_float2(0.f, 0.f);
            else
                rx[v] = make_float2(in ? xfr[(size_t)(k - d) * N + j] : 0.f, 0.f);
        }
    };
    auto store_tile = [&]() {
#pragma unroll
        for (int v = 0; v < AV; ++v) {
            const int t = threadIdx.x + v * MV_THREADS;
            const int i = t / (TJ / 4), jq = 4 * (t % (TJ / 4));
            As[jq][i] = ra[v].x;
            As[jq + 1][i] = ra[v].y;
            As[jq + 2][i] = ra[v].z;
            As[jq + 3][i] = ra[v].w;
        }
#pragma unroll
        for (int v = 0; v < XV; ++v) {
            const int t = threadIdx.x + v * MV_THREADS;
            Xs[t / TK][t % TK] = make_float4(rx[v].x, rx[v].x, rx[v].y, rx[v].y);
        }
    };

    load_tile(0);
    for (int it = 0; it < n_it; ++it) {
        store_tile();
        __syncthreads();
        if (it + 1 < n_it) load_tile(it + 1);
#pragma unroll 4
        for (int jj = 0; jj < TJ; ++jj) {
            const float4 xv = Xs[jj][tx];
            const float2 xh = make_float2(xv.x, xv.y), xl = make_float2(xv.z, xv.w);
            const float2 nxh = make_float2(-xv.x, -xv.y);
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[jj][ty * RPT]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[jj][ty * RPT + 4]);
            df_acc2<SPLIT>(make_float2(a0.x, a0.y), xh, nxh, xl, hi[0], lo[0]);
            df_acc2<SPLIT>(make_float2(a0.z, a0.w), xh, nxh, xl, hi[1], lo[1]);
            df_acc2<SPLIT>(make_float2(a1.x, a1.y), xh, nxh, xl, hi[2], lo[2]);
            df_acc2<SPLIT>(make_float2(a1.z, a1.w), xh, nxh, xl, hi[3], lo[3]);
        }
        __syncthreads();
    }
    const int k = k0 + tx;
    if (k >= n_steps) return;
    double *pr = part + (((size_t)dr * nrhs + r) * n_steps + k) * E;
#pragma unroll
    for (int i = 0; i < RPT / 2; ++i) {
        const int l = l0 + ty * RPT + 2 * i;
        if (l < E) pr[l] = (double)hi[i].x + (double)lo[i].x;
        if (l + 1 < E) pr[l + 1] = (double)hi[i].y + (double)lo[i].y;
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
    for (int dr = 0; dr * DF_TD <= k; ++dr) s += part[dr * total + idx];
    if (mode == DF_RESIDUAL)
        y[idx] = f[idx] - s;
    else
        y[idx] = beta == 0.0 ? s : fma(beta, y[idx], s);
}

size_t toeplitz_df_bytes(int64_t E, int32_t n_steps, int32_t nrhs) {
    return toeplitz_df_rect_bytes(E, E, n_steps, nrhs);
}

size_t toeplitz_df_rect_bytes(int64_t E, int64_t N, int32_t n_steps, int32_t nrhs) {
    return df_partial_bytes(E, n_steps, nrhs) + align256((size_t)nrhs * n_steps * N * sizeof(float2));
}

// y = A x for blocks of E rows and N columns (x: [nrhs][n_steps][N], y and
// f: [nrhs][n_steps][E]).
static stb_status toeplitz_df_run(const float *A, int64_t E, int64_t N, int32_t n_steps,
                                  int32_t nrhs, const double *x, const float *xf, int mode,
                                  const double *f, double beta, double *y, void *scratch,
                                  cudaStream_t s) {
    double *part = static_cast<double *>(scratch);
    float2 *xs = reinterpret_cast<float2 *>(static_cast<char *>(scratch) +
                                            df_partial_bytes(E, n_steps, nrhs));
    const size_t total = (size_t)nrhs * n_steps * E, total_x = (size_t)nrhs * n_steps * N;
    stb_status st;
    if (x) {
        count_launch(s);
        k_split<<<(unsigned)((total_x + 255) / 256), 256, 0, s>>>(x, total_x, xs);
        if ((st = check_launch("k_split"))) return st;
    }
    int n_kt = (n_steps + TK - 1) / TK, n_dr = (n_steps + DF_TD - 1) / DF_TD;
    dim3 grid((unsigned)((E + TM - 1) / TM), (unsigned)(n_kt * nrhs), (unsigned)n_dr);
    const bool vec = N % 4 == 0 && reinterpret_cast<uintptr_t>(A) % 16 == 0;
    const auto kern = x ? (vec ? k_toeplitz_df_partial<true, true> : k_toeplitz_df_partial<false, true>)
                        : (vec ? k_toeplitz_df_partial<true, false>
                               : k_toeplitz_df_partial<false, false>);
    count_launch(s);
    kern<<<grid, MV_THREADS, 0, s>>>(A, (int)E, (int)N, n_steps, nrhs, xs, xf, part);
    if ((st = check_launch("k_toeplitz_df_partial"))) return st;
    count_launch(s);
    k_toeplitz_df_reduce<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(part, (int)E, n_steps, nrhs,
                                                                         mode, f, beta, y);
    return check_launch("k_toeplitz_df_reduce");
}

stb_status toeplitz_df(const float *A, int64_t E, int32_t n_steps, int32_t nrhs, const double *x,
                       int mode, const double *f, double beta, double *y, void *scratch,
                       cudaStream_t s) {
    return toeplitz_df_run(A, E, E, n_steps, nrhs, x, nullptr, mode, f, beta, y, scratch, s);
}

stb_status toeplitz_df_f32x(const float *A, int64_t E, int32_t n_steps, int32_t nrhs,
                            const float *x, int mode, const double *f, double beta, double *y,
                            void *scratch, cudaStream_t s) {
    return toeplitz_df_run(A, E, E, n_steps, nrhs, nullptr, x, mode, f, beta, y, scratch, s);
}

stb_status toeplitz_df_rect(const float *A, int64_t E, int64_t N, int32_t n_steps, int32_t nrhs,
                            const double *x, double *y, void *scratch, cudaStream_t s) {
    return toeplitz_df_run(A, E, N, n_steps, nrhs, x, nullptr, DF_AXPBY, nullptr, 0.0, y, scratch,
                           s);
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
    case STB_ARITH_SPLIT: *bytes = 256 + toeplitz_split_bytes(E, n_steps, nrhs); return STB_OK;
    default:
        return fail(STB_ERR_INVALID_ARG, "arith must be STB_ARITH_FP64, _DF, _TF32 or _SPLIT");
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
        return fail(STB_ERR_INVALID_ARG,
                    "STB_ARITH_DF, STB_ARITH_TF32 and STB_ARITH_SPLIT need STB_STORE_F32 blocks");
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
    if (arith == STB_ARITH_SPLIT)
        return toeplitz_split((const float *)A, E, n_steps, nrhs, x, DF_AXPBY, nullptr, beta, y,
                              scratch, status_word(ws), s);
    return toeplitz_tc((const float *)A, E, n_steps, nrhs, x, beta, y, scratch, status_word(ws), s);
}
