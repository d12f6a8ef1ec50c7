// stb_solve.cu -- solution of the block lower-triangular Toeplitz system
// V_h w = f of the Dirichlet problem (eq. V_mat, Sec. 3.4) by block forward
// substitution in time:
//     w^k = (V^0)^{-1} ( f^k - sum_{d=1}^{k} V^d w^{k-d} ),  k = 0..E_t-1.
// V^0 is symmetric positive definite; it is factorised once, V^0 = L L^T, by
// a right-looking blocked Cholesky (64 x 64 tiles), L is inverted blockwise
// and (V^0)^{-1} = L^{-T} L^{-1} formed explicitly.  Steps are grouped in
// panels of 8: the history from earlier panels is one blocked product per
// panel, and the panel's steps -- the history sum inside the panel (reads
// the blocks V^d once, all right-hand sides together) and w^k = (V^0)^{-1} r
// -- run in one cooperative launch with grid barriers between the phases.
//
// FP64 precision: everything in FP64.
// Mixed precision: the factorisation and the march run in FP32 and are wrapped
// in iterative refinement,  w <- w + march(f - V_h w),  whose residual is
// updated as r <- r - V_h delta with the split-operand tensor-core product
// (bf16 digit slices of the stored FP32 blocks and of the FP32 correction
// delta, exact FP32 sums per chunk, about 44 bits), so that no O(E^2 E_t^2)
// work runs on the scarce FP64 pipe.  The refinement stops at
// ||r|| <= 1e-10 ||f||.
#include <algorithm>
#include <cmath>
#include <vector>

#include "stb_dense.h"
#include "stb_grid.cuh"
#include "stb_internal.h"
#include "stb_toeplitz.h"

namespace stb {

constexpr int NB = 64;

template <class S, class T>
__global__ void k_copy_convert(const S *__restrict__ src, size_t n, T *__restrict__ dst) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (T)src[i];
}

// ---------------------------------------------- blocked Cholesky ---
// V^0 = L L^T by 64 x 64 tiles, right-looking, all panels in one cooperative
// launch: for each tile column kb, (1) CTA 0 factorises the diagonal tile,
// (2) the tiles below it are solved against it, (3) the trailing tiles are
// updated, grid barriers between the phases.  L is read with __ldcg (other
// CTAs wrote it in this launch).

// Cholesky of diagonal tile kb (updates from the left already applied).
// Each thread keeps its elements of the tile's lower triangle (linear index
// tid + 256 u) in registers through all 64 column steps; step c subtracts
// a_ic a_jc / a_cc from the trailing elements (j > c) with the raw column c,
// whose owners published it in shared memory after its last update, so a
// step needs one barrier.  At the end a_ij / sqrt(a_jj) (i > j) and
// sqrt(a_jj) are the entries of L.
constexpr int POTRF_THREADS = 256;
constexpr int POTRF_SLOTS = (NB * (NB + 1) / 2 + POTRF_THREADS - 1) / POTRF_THREADS;
template <class T>
__device__ void potrf_tile(T *__restrict__ L, int E, int kb, int32_t *__restrict__ status,
                           T (*col)[NB], T *piv) {
    const int b0 = kb * NB, n = min(NB, E - b0);
    T val[POTRF_SLOTS];
    int ri[POTRF_SLOTS], ci[POTRF_SLOTS];
#pragma unroll
    for (int u = 0; u < POTRF_SLOTS; ++u) {
        const int t = threadIdx.x + POTRF_THREADS * u;
        int i = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);  // row of the t-th lower element
        while ((i + 1) * (i + 2) / 2 <= t) ++i;
        while (i * (i + 1) / 2 > t) --i;
        const int j = t - i * (i + 1) / 2;
        const bool in = t < NB * (NB + 1) / 2 && i < n;
        ri[u] = in ? i : NB;  // NB: not an element of this tile
        ci[u] = in ? j : NB;
        val[u] = in ? __ldcg(L + (size_t)(b0 + i) * E + b0 + j) : (T)0;
        if (in && j == 0) col[0][i] = val[u];
    }
    __syncthreads();
    for (int c = 0; c < n; ++c) {
        const T(*cc)[NB] = col + (c & 1);
        T d = (*cc)[c];
        if (!(d > (T)0)) {
            if (threadIdx.x == 0) atomicCAS(status, 0, STB_ERR_NOT_SPD);
            d = (T)1;
        }
        if (threadIdx.x == 0) piv[c] = d;
        const T inv = (T)1 / d;
#pragma unroll
        for (int u = 0; u < POTRF_SLOTS; ++u) {
            if (ci[u] > c && ci[u] < NB) {
                val[u] = fma(-(*cc)[ri[u]] * inv, (*cc)[ci[u]], val[u]);
                if (ci[u] == c + 1) col[(c + 1) & 1][ri[u]] = val[u];
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < POTRF_SLOTS; ++u) {
        const int i = ri[u], j = ci[u];
        if (i < NB) {
            const T sj = sqrt(piv[j]);
            L[(size_t)(b0 + i) * E + b0 + j] = i == j ? sj : val[u] / sj;
        }
    }
    for (int t = threadIdx.x; t < n * n; t += POTRF_THREADS) {  // the strict upper triangle
        const int i = t / n, j = t % n;
        if (j > i) L[(size_t)(b0 + i) * E + b0 + j] = (T)0;
    }
}

// Panel: L_ik = A_ik L_kk^{-T} for tile row i = kb + 1 + bi.  Four threads
// per row (blockDim 256), each holding the columns q, q+4, .. of its row in
// registers; column c is solved by its owner and broadcast to the other
// three lanes by a shuffle, and every later column is updated at once
// (independent FMAs instead of one dependent chain per row).
template <class T>
__device__ void trsm_tile(T *__restrict__ L, int E, int kb, int bi, T (*Lk)[NB + 1]) {
    const int b0 = kb * NB, n = min(NB, E - b0);
    const int i0 = (kb + 1 + bi) * NB, mrows = min(NB, E - i0);
    const int row = threadIdx.x >> 2, q = threadIdx.x & 3;
    const unsigned lane = threadIdx.x & 31;
    __syncthreads();  // the shared tile of the previous task is consumed
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
        int i = t / NB, j = t % NB;
        Lk[i][j] = (i < n && j < n) ? __ldcg(L + (size_t)(b0 + i) * E + b0 + j) : (T)0;
    }
    T v[NB / 4];
#pragma unroll
    for (int j = 0; j < NB / 4; ++j) {
        const int c = 4 * j + q;
        v[j] = (row < mrows && c < n) ? __ldcg(L + (size_t)(i0 + row) * E + b0 + c) : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NB; ++c) {
        if (c >= n) break;
        const int oj = c >> 2;
        T x = v[oj] / Lk[c][c];  // meaningful on the owner lane (q == c % 4)
        x = __shfl_sync(0xffffffffu, x, (int)((lane & ~3u) | (unsigned)(c & 3)));
        if (q == (c & 3)) v[oj] = x;
#pragma unroll
        for (int j = oj; j < NB / 4; ++j)
            if (4 * j + q > c) v[j] = fma(-x, Lk[4 * j + q][c], v[j]);
    }
#pragma unroll
    for (int j = 0; j < NB / 4; ++j) {
        const int c = 4 * j + q;
        if (row < mrows && c < n) L[(size_t)(i0 + row) * E + b0 + c] = v[j];
    }
}

// 64x64 tile product helper: acc (4x4 per thread, 256 threads) +=
// P (rows of the tile) * Q^T, both read from global in 32-wide chunks (CG:
// through L2 only, for data other CTAs of the launch wrote).
template <class T> struct TileAcc {
    T v[4][4];
};

template <class T, bool CG = false>
__device__ __forceinline__ void tile_mma_abt(TileAcc<T> &acc, const T *P, size_t ldp, int prow,
                                             int pcol, const T *Q, size_t ldq, int qrow, int qcol,
                                             int E, int kn, T (*Ps)[33], T (*Qs)[33]) {
    // acc[i][j] += sum_k P[prow+i][pcol+k] * Q[qrow+j][qcol+k], k < kn
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    for (int k0 = 0; k0 < kn; k0 += 32) {
        for (int t = threadIdx.x; t < NB * 32; t += blockDim.x) {
            int r = t / 32, kk = t % 32;
            int pr = prow + r, qr = qrow + r, pc = pcol + k0 + kk, qc = qcol + k0 + kk;
            const T *pp = P + (size_t)pr * ldp + pc, *qp = Q + (size_t)qr * ldq + qc;
            if constexpr (CG) {
                Ps[r][kk] = (pr < E && k0 + kk < kn) ? __ldcg(pp) : (T)0;
                Qs[r][kk] = (qr < E && k0 + kk < kn) ? __ldcg(qp) : (T)0;
            } else {
                Ps[r][kk] = (pr < E && k0 + kk < kn) ? *pp : (T)0;
                Qs[r][kk] = (qr < E && k0 + kk < kn) ? *qp : (T)0;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 32; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = Ps[4 * ty + u][kk];
                b[u] = Qs[4 * tx + u][kk];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc.v[u][v] = fma(a[u], b[v], acc.v[u][v]);
        }
        __syncthreads();
    }
}

// Trailing update A_ij -= L_ik L_jk^T for the t-th tile pair kb < j <= i.
template <class T>
__device__ void syrk_tile(T *__restrict__ L, int E, int kb, int t, T (*Ps)[33], T (*Qs)[33]) {
    int ii = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
    while (ii * (ii + 1) / 2 > t) --ii;
    const int jj = t - ii * (ii + 1) / 2;
    const int i0 = (kb + 1 + ii) * NB, j0 = (kb + 1 + jj) * NB, b0 = kb * NB;
    const int kn = min(NB, E - b0);
    TileAcc<T> acc;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc.v[u][v] = (T)0;
    __syncthreads();  // the shared tiles of the previous task are consumed
    tile_mma_abt<T, true>(acc, L, E, i0, b0, L, E, j0, b0, E, kn, Ps, Qs);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    for (int u = 0; u < 4; ++u)
        for (int v = 0; v < 4; ++v) {
            int r = i0 + 4 * ty + u, c = j0 + 4 * tx + v;
            if (r < E && c < E) L[(size_t)r * E + c] = __ldcg(L + (size_t)r * E + c) - acc.v[u][v];
        }
}

template <class T>
constexpr size_t potrf_smem() {
    // the larger of the phases' tiles: L_kk of the panel solve, or the two
    // operand chunks of the trailing update
    return (NB * (NB + 1) > 2 * NB * 33 ? (size_t)NB * (NB + 1) : (size_t)2 * NB * 33) * sizeof(T);
}

template <class T>
__global__ void __launch_bounds__(256) k_potrf_coop(T *__restrict__ L, int E, int nb,
                                                    int32_t *__restrict__ status, unsigned *bar) {
    extern __shared__ __align__(16) unsigned char fsm[];
    __shared__ T col[2][NB], piv[NB];
    T(*T1)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(fsm);
    T(*Ps)[33] = reinterpret_cast<T(*)[33]>(fsm);
    T(*Qs)[33] = reinterpret_cast<T(*)[33]>(fsm + (size_t)NB * 33 * sizeof(T));
    // look-ahead: in the update phase of column kb, CTA 0 first updates the
    // next diagonal tile (pair 0) and factorises it while the other CTAs
    // update the rest, so a column costs two grid barriers
    if (blockIdx.x == 0) potrf_tile<T>(L, E, 0, status, col, piv);
    if (!grid_barrier(bar, status)) return;
    for (int kb = 0; kb < nb; ++kb) {
        const int m = nb - kb - 1;
        if (m == 0) break;
        for (int bi = blockIdx.x; bi < m; bi += gridDim.x) trsm_tile<T>(L, E, kb, bi, T1);
        if (!grid_barrier(bar, status)) return;
        const int tiles = m * (m + 1) / 2;
        if (blockIdx.x == 0) {
            syrk_tile<T>(L, E, kb, 0, Ps, Qs);
            __syncthreads();  // the CTA's own updates of the tile, read back below
            potrf_tile<T>(L, E, kb + 1, status, col, piv);
        }
        const int first = gridDim.x > 1 ? 1 : 0, step = gridDim.x > 1 ? gridDim.x - 1 : 1;
        if (gridDim.x == 1 || blockIdx.x > 0)
            for (int t = 1 + (int)blockIdx.x - first; t < tiles; t += step)
                syrk_tile<T>(L, E, kb, t, Ps, Qs);
        if (!grid_barrier(bar, status)) return;
    }
}

// (V^0)^{-1} = L^{-T} L^{-1} from U = L^{-T} (upper triangular):
// M_IJ = sum_{c >= max(I,J)} U_Ic U_Jc^T, tile pairs I >= J, both halves written.
template <class T>
__global__ void __launch_bounds__(256) k_inverse_spd(const T *__restrict__ U, T *__restrict__ M,
                                                     int E) {
    __shared__ T Ps[NB][33], Qs[NB][33];
    const int t = blockIdx.x;
    int ii = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
    while (ii * (ii + 1) / 2 > t) --ii;
    const int jj = t - ii * (ii + 1) / 2;
    const int i0 = ii * NB, j0 = jj * NB;
    TileAcc<T> acc;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc.v[u][v] = (T)0;
    tile_mma_abt<T>(acc, U, E, i0, i0, U, E, j0, i0, E, E - i0, Ps, Qs);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    for (int u = 0; u < 4; ++u)
        for (int v = 0; v < 4; ++v) {
            const int r = i0 + 4 * ty + u, c = j0 + 4 * tx + v;
            if (r < E && c < E) {
                M[(size_t)r * E + c] = acc.v[u][v];
                M[(size_t)c * E + r] = acc.v[u][v];
            }
        }
}

// Inverse of every diagonal tile of L (lower triangular), in parallel.
template <class T>
__global__ void __launch_bounds__(64) k_trtri_diag(const T *__restrict__ L, T *__restrict__ Li,
                                                   int E) {
    __shared__ T Tt[NB][NB + 1];
    __shared__ T X[NB][NB + 1];
    const int b0 = blockIdx.x * NB, n = min(NB, E - b0);
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
        int i = t / NB, j = t % NB;
        Tt[i][j] = (i < n && j < n) ? L[(size_t)(b0 + i) * E + b0 + j] : (T)0;
        X[i][j] = (T)0;
    }
    __syncthreads();
    const int c = threadIdx.x;  // column of the inverse
    if (c < n) {
        for (int i = c; i < n; ++i) {
            T x = (i == c) ? (T)1 : (T)0;
            for (int m = c; m < i; ++m) x = fma(-Tt[i][m], X[m][c], x);
            X[i][c] = x / Tt[i][i];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        int i = t / n, j = t % n;
        Li[(size_t)(b0 + i) * E + b0 + j] = X[i][j];
    }
}

// Batched tile product for the recursive inversion of L: task (i, j, mlo, mhi)
// writes tile C_ij = alpha sum_{m=mlo}^{mhi} A_im B_mj (tiles of NB x NB).
template <class T>
__global__ void __launch_bounds__(256)
k_tile_gemm(const int4 *__restrict__ tasks, const T *__restrict__ A, const T *__restrict__ B,
            T *__restrict__ C, int E, T alpha) {
    __shared__ T Ps[NB][33], Qs[NB][33];
    const int4 tk = tasks[blockIdx.x];
    const int i0 = tk.x * NB, j0 = tk.y * NB;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    TileAcc<T> acc;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc.v[u][v] = (T)0;
    for (int m = tk.z; m <= tk.w; ++m) {
        const int m0 = m * NB;
        for (int k0 = 0; k0 < NB; k0 += 32) {
            for (int t = threadIdx.x; t < NB * 32; t += blockDim.x) {
                const int r = t / 32, kk = t % 32, gr = i0 + r, gk = m0 + k0 + kk;
                Ps[r][kk] = (gr < E && gk < E) ? A[(size_t)gr * E + gk] : (T)0;
                // B rows read along their columns (coalesced), stored transposed
                const int c = t % NB, kq = t / NB, gq = m0 + k0 + kq, gc = j0 + c;
                Qs[c][kq] = (gq < E && gc < E) ? B[(size_t)gq * E + gc] : (T)0;
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < 32; ++kk) {
                T a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    a[u] = Ps[4 * ty + u][kk];
                    b[u] = Qs[4 * tx + u][kk];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc.v[u][v] = fma(a[u], b[v], acc.v[u][v]);
            }
            __syncthreads();
        }
    }
    for (int u = 0; u < 4; ++u)
        for (int v = 0; v < 4; ++v) {
            const int r = i0 + 4 * ty + u, c = j0 + 4 * tx + v;
            if (r < E && c < E) C[(size_t)r * E + c] = alpha * acc.v[u][v];
        }
}

// Task lists of the recursive inversion of the lower-triangular tile matrix
// L (nb x nb tiles): a node [a, b) with children [a, c), [c, b) whose
// inverses are known gets  Li_21 = -Li_22 (L_21 Li_11),  as two batched
// products per tree level (deepest level first):
//   phase 1: W_ij = sum_{m=j}^{c-1} L_im Li_mj      (i in [c,b), j in [a,c))
//   phase 2: Li_ij = -sum_{m=c}^{i} Li_im W_mj
struct InvLevel {
    std::vector<int4> p1, p2;
};

static void inv_tasks(int a, int b, int depth, std::vector<InvLevel> &lv) {
    if (b - a < 2) return;
    const int c = a + (b - a) / 2;
    inv_tasks(a, c, depth + 1, lv);
    inv_tasks(c, b, depth + 1, lv);
    if ((int)lv.size() <= depth) lv.resize(depth + 1);
    for (int i = c; i < b; ++i)
        for (int j = a; j < c; ++j) {
            lv[depth].p1.push_back(make_int4(i, j, j, c - 1));
            lv[depth].p2.push_back(make_int4(i, j, c, i));
        }
}

// The same task lists written on the device (no host copy, so the
// factorisation can be captured into a CUDA graph): per tree depth, the
// phase-1 tasks at off[depth] and the phase-2 tasks cnt[depth] later, nodes
// of one depth in the left-to-right order of the host recursion above.
constexpr int INV_MAX_DEPTH = 32;
struct InvOffs {
    int off[INV_MAX_DEPTH], cnt[INV_MAX_DEPTH];
};

__global__ void k_inv_tasks(int nb, int n_levels, InvOffs o, int4 *out) {
    for (int d = 0; d < n_levels; ++d) {
        int fill = 0;
        // nodes of depth d left to right: paths of d halving choices, first
        // choice in the highest bit (0 = left half)
        for (long long path = 0; path < (1LL << d); ++path) {
            int a = 0, b = nb;
            bool ok = true;
            for (int k = d - 1; k >= 0 && ok; --k) {
                if (b - a < 2) {
                    ok = false;
                } else {
                    const int c = a + (b - a) / 2;
                    if ((path >> k) & 1) a = c;
                    else b = c;
                }
            }
            if (!ok || b - a < 2) continue;
            const int c = a + (b - a) / 2;
            for (int i = c; i < b; ++i)
                for (int j = a; j < c; ++j, ++fill) {
                    out[o.off[d] + fill] = make_int4(i, j, j, c - 1);
                    out[o.off[d] + o.cnt[d] + fill] = make_int4(i, j, c, i);
                }
        }
    }
}

static size_t inv_task_count(int nb) {
    std::vector<InvLevel> lv;
    inv_tasks(0, nb, 0, lv);
    size_t n = 0;
    for (auto &l : lv) n += l.p1.size() + l.p2.size();
    return n;
}

template <class T>
__global__ void k_transpose(const T *__restrict__ A, T *__restrict__ B, int E) {
    __shared__ T t[32][33];
    int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 32 + threadIdx.y;
    for (int k = 0; k < 32; k += 8)
        if (x < E && y + k < E) t[threadIdx.y + k][threadIdx.x] = A[(size_t)(y + k) * E + x];
    __syncthreads();
    x = blockIdx.y * 32 + threadIdx.x;
    y = blockIdx.x * 32 + threadIdx.y;
    for (int k = 0; k < 32; k += 8)
        if (x < E && y + k < E) B[(size_t)(y + k) * E + x] = t[threadIdx.x][threadIdx.y + k];
}

constexpr int MAXR = 8;  // right-hand sides per pass of the march kernels

// Far history of a panel of PB steps k = kp + c (c < nb): all contributions
// of the steps before the panel,
//   sum_{d : 0 <= k-d < kp} V^d[l,:] x_r^{k-d},
// a skinny product (PB columns per right-hand side) over the blocks
// d = 1..kp+nb-1.  Register tiling: a warp owns R rows, a lane four
// consecutive columns j, so one vector load of V feeds 4 x PB FMAs per row and
// one load of x feeds R x 4.  The block range is cut into gridDim.y slices of
// dz blocks whose partial sums k_far_reduce adds up.
constexpr int PB = 8;
constexpr int FAR_NZ = 16;  // at most this many slices
template <class T, int PR>
constexpr int far_rows_per_warp() { return (sizeof(T) == 4 ? 4 : 2) / PR; }

// four consecutive elements p[0..3] as T; VEC: p is 16-byte aligned and all
// four are in range, else only the first `left` of them are
template <class S, class T, bool VEC>
__device__ __forceinline__ void load4(const S *__restrict__ p, int left, T v[4]) {
    if constexpr (VEC && sizeof(S) == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = (T)q.x, v[1] = (T)q.y, v[2] = (T)q.z, v[3] = (T)q.w;
    } else if constexpr (VEC) {
        const double2 a = reinterpret_cast<const double2 *>(p)[0];
        const double2 b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = (T)a.x, v[1] = (T)a.y, v[2] = (T)b.x, v[3] = (T)b.y;
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = u < left ? (T)p[u] : (T)0;
    }
}

// part[z][r][c][l] = slice z's share of the far history (T)
template <class AT, class T, int PR, bool VEC>
__global__ void __launch_bounds__(256, 2)
k_history_far(const AT *__restrict__ V, int E, int n_steps, int nrhs, int kp, int nb, int dz,
              const T *__restrict__ x, T *__restrict__ part) {
    constexpr int FAR_R = far_rows_per_warp<T, PR>();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int l0 = (blockIdx.x * 8 + warp) * FAR_R;
    const int dlo = 1 + (int)blockIdx.y * dz, dhi = min(dlo + dz, kp + nb);
    const size_t EE = (size_t)E * E, SE = (size_t)n_steps * E;
    for (int r0 = 0; r0 < nrhs; r0 += PR) {
        T acc[PR][FAR_R][PB];
#pragma unroll
        for (int r = 0; r < PR; ++r)
#pragma unroll
            for (int i = 0; i < FAR_R; ++i)
#pragma unroll
                for (int c = 0; c < PB; ++c) acc[r][i][c] = (T)0;
        for (int d = dlo; d < dhi; ++d) {
            // columns c with 0 <= kp + c - d < kp (non-empty for 1 <= d < kp + nb, kp >= 1)
            const int cl = max(kp, d) - kp, ch = min(kp + nb - 1, kp - 1 + d) - kp;
            const AT *Vd = V + (size_t)d * EE;
#pragma unroll 1
            for (int j = 4 * lane; j < E; j += 128) {
                T v[FAR_R][4];
#pragma unroll
                for (int i = 0; i < FAR_R; ++i)  // rows past E re-read row E-1, never stored
                    load4<AT, T, VEC>(Vd + (size_t)min(l0 + i, E - 1) * E + j, E - j, v[i]);
#pragma unroll
                for (int c = 0; c < PB; ++c) {
                    if (c < cl || c > ch) continue;
#pragma unroll
                    for (int r = 0; r < PR; ++r) {
                        if (r0 + r >= nrhs) continue;
                        T xv[4];
                        load4<T, T, VEC>(x + (size_t)(r0 + r) * SE + (size_t)(kp + c - d) * E + j,
                                         E - j, xv);
#pragma unroll
                        for (int i = 0; i < FAR_R; ++i)
#pragma unroll
                            for (int u = 0; u < 4; ++u) acc[r][i][c] = fma(v[i][u], xv[u], acc[r][i][c]);
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < PR; ++r)
#pragma unroll
            for (int i = 0; i < FAR_R; ++i)
#pragma unroll
                for (int c = 0; c < PB; ++c) {
                    T a = acc[r][i][c];
                    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                    if (lane == 0 && r0 + r < nrhs && c < nb && l0 + i < E)
                        part[(((size_t)blockIdx.y * nrhs + r0 + r) * PB + c) * E + l0 + i] = a;
                }
    }
}

// hv_r[c][l] = f_r^{kp+c}[l] - sum_z part[z][r][c][l]  (c < nb)
template <class T>
__global__ void k_far_reduce(const T *__restrict__ part, int nz, int E, int n_steps, int nrhs, int kp,
                             int nb, const double *__restrict__ f, double *__restrict__ hv) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)nrhs * nb * E) return;
    const int l = (int)(i % E), c = (int)((i / E) % nb), r = (int)(i / ((size_t)E * nb));
    double s = 0.0;
    for (int z = 0; z < nz; ++z) s += (double)part[(((size_t)z * nrhs + r) * PB + c) * E + l];
    hv[((size_t)r * PB + c) * E + l] = f[(size_t)r * n_steps * E + (size_t)(kp + c) * E + l] - s;
}

// ------------------------------------------------ the steps of a panel ---
// One cooperative launch per panel of PB steps k = kp + c (c < nb):
//   phase 1: rv_r = hv_r^c - sum_{d=1}^{c} V^d x_r^{k-d}   (history inside the panel)
//   grid barrier
//   phase 2: x_r^k = (V^0)^{-1} rv_r
//   grid barrier (not after the last step)
// A CTA owns blocks of 8 warps x RW rows (grid-stride); the vectors of a
// phase (x^{k-d}, or rv) are staged in shared memory chunk by chunk by the
// whole CTA, read from L2 (__ldcg: other CTAs wrote them in this launch), and
// each warp streams its rows of the matrix against them, four consecutive
// columns per lane and load, MP_MR right-hand sides per pass.
constexpr int MP_THREADS = 256;
// rows per warp RW: 2, or 3 for FP32 blocks and vectors when the 24-row
// blocks still give every SM one (fewer, larger blocks then stream the
// matrices faster: two 256-thread CTAs per SM at about 126 registers)
template <class AT, class T, int RW>
constexpr int mp_min_ctas() { return sizeof(AT) == 4 && sizeof(T) == 4 && RW == 3 ? 2 : 1; }
constexpr int MP_MR = 8;  // right-hand sides per pass
// columns per staged chunk: 16 (FP64: 8) per lane and row, 2 KB of an FP32 row
template <class AT, class T>
constexpr int mp_chunk() { return (sizeof(AT) == 8 || sizeof(T) == 8) ? 256 : 512; }

// four consecutive T from L2 (bypassing L1), VEC: 16-byte aligned and in range
template <class T, bool VEC>
__device__ __forceinline__ void load4_cg(const T *p, int left, T v[4]) {
    if constexpr (VEC && sizeof(T) == 4) {
        const float4 q = __ldcg(reinterpret_cast<const float4 *>(p));
        v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
    } else if constexpr (VEC) {
        const double2 a = __ldcg(reinterpret_cast<const double2 *>(p));
        const double2 b = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
        v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = u < left ? __ldcg(p + u) : (T)0;
    }
}

// acc[i][r] += sum_j Mat[l0 + i][j] vec_r[j] (this lane's columns; rows past
// E re-read row E-1 and are never stored), vec_r = vec + r vstride, r < nr.
template <class MT, class T, int JC, int RW, bool VEC>
__device__ __forceinline__ void mp_pass(const MT *__restrict__ mat, int E, int l0, const T *vec,
                                        size_t vstride, int nr, T *stage, T (&acc)[RW][MP_MR]) {
    constexpr int G = JC / 128;  // groups of four columns per lane
    const int lane = threadIdx.x & 31;
    for (int j0 = 0; j0 < E; j0 += JC) {
        const int jn = min(JC, E - j0);
        __syncthreads();  // the previous chunk is consumed
        for (int t = threadIdx.x; t < nr * (JC / 4); t += MP_THREADS) {
            const int r = t / (JC / 4), jj = 4 * (t % (JC / 4));
            T v[4] = {(T)0, (T)0, (T)0, (T)0};
            if (jj < jn) load4_cg<T, VEC>(vec + r * vstride + j0 + jj, jn - jj, v);
#pragma unroll
            for (int u = 0; u < 4; ++u) stage[r * JC + jj + u] = v[u];
        }
        __syncthreads();
        T m[RW][G][4];
#pragma unroll
        for (int i = 0; i < RW; ++i)
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int jj = 128 * g + 4 * lane;
#pragma unroll
                for (int u = 0; u < 4; ++u) m[i][g][u] = (T)0;
                if (jj < jn)
                    load4<MT, T, VEC>(mat + (size_t)min(l0 + i, E - 1) * E + j0 + jj, jn - jj,
                                      m[i][g]);
            }
#pragma unroll
        for (int r = 0; r < MP_MR; ++r) {
            if (r >= nr) break;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const T *xs = stage + r * JC + 128 * g + 4 * lane;
                T xv[4];
                if constexpr (sizeof(T) == 4) {
                    const float4 q = *reinterpret_cast<const float4 *>(xs);
                    xv[0] = q.x, xv[1] = q.y, xv[2] = q.z, xv[3] = q.w;
                } else {
                    const double2 a = reinterpret_cast<const double2 *>(xs)[0];
                    const double2 b = reinterpret_cast<const double2 *>(xs)[1];
                    xv[0] = a.x, xv[1] = a.y, xv[2] = b.x, xv[3] = b.y;
                }
#pragma unroll
                for (int i = 0; i < RW; ++i)
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc[i][r] = fma(m[i][g][u], xv[u], acc[i][r]);
            }
        }
    }
}

// sums over the warp; lane i MP_MR + r ends up holding (row i, rhs r)
template <class T, int RW>
__device__ __forceinline__ T mp_reduce(T (&acc)[RW][MP_MR]) {
    const int lane = threadIdx.x & 31;
    T mine = (T)0;
#pragma unroll
    for (int i = 0; i < RW; ++i)
#pragma unroll
        for (int r = 0; r < MP_MR; ++r) {
            T a = acc[i][r];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == i * MP_MR + r) mine = a;
        }
    return mine;
}

template <class AT, class T, int RW, bool VEC>
__global__ void __launch_bounds__(MP_THREADS, mp_min_ctas<AT, T, RW>())
k_march_panel(const AT *__restrict__ V, const T *__restrict__ Minv, int E, int n_steps, int nrhs,
              int kp, int nb, const double *__restrict__ hv, T *rv, T *x, unsigned *bar,
              int32_t *status) {
    constexpr int JC = mp_chunk<AT, T>();
    static_assert(RW * MP_MR <= 32, "one lane per (row, right-hand side)");
    __shared__ __align__(16) T stage[MP_MR * JC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rows_cta = 8 * RW, n_rb = (E + rows_cta - 1) / rows_cta;
    const size_t EE = (size_t)E * E, SE = (size_t)n_steps * E;
    const int li = lane / MP_MR, lr = lane % MP_MR;  // this lane's (row, rhs) of a pass
    for (int c = 0; c < nb; ++c) {
        const int k = kp + c;
        for (int rb = blockIdx.x; rb < n_rb; rb += gridDim.x) {
            const int l0 = rb * rows_cta + warp * RW;
            for (int r0 = 0; r0 < nrhs; r0 += MP_MR) {
                const int nr = min(MP_MR, nrhs - r0);
                T acc[RW][MP_MR];
#pragma unroll
                for (int i = 0; i < RW; ++i)
#pragma unroll
                    for (int r = 0; r < MP_MR; ++r) acc[i][r] = (T)0;
                for (int d = 1; d <= c; ++d)
                    mp_pass<AT, T, JC, RW, VEC>(V + d * EE, E, l0, x + r0 * SE + (size_t)(k - d) * E, SE,
                                            nr, stage, acc);
                const T a = mp_reduce(acc);
                const int l = l0 + li;
                if (li < RW && lr < nr && l < E)
                    rv[(size_t)(r0 + lr) * E + l] =
                        (T)(hv[((size_t)(r0 + lr) * PB + c) * E + l] - (double)a);
            }
        }
        if (!grid_barrier(bar, status)) return;
        for (int rb = blockIdx.x; rb < n_rb; rb += gridDim.x) {
            const int l0 = rb * rows_cta + warp * RW;
            for (int r0 = 0; r0 < nrhs; r0 += MP_MR) {
                const int nr = min(MP_MR, nrhs - r0);
                T acc[RW][MP_MR];
#pragma unroll
                for (int i = 0; i < RW; ++i)
#pragma unroll
                    for (int r = 0; r < MP_MR; ++r) acc[i][r] = (T)0;
                mp_pass<T, T, JC, RW, VEC>(Minv, E, l0, rv + (size_t)r0 * E, E, nr, stage, acc);
                const T a = mp_reduce(acc);
                const int l = l0 + li;
                if (li < RW && lr < nr && l < E) x[(size_t)(r0 + lr) * SE + (size_t)k * E + l] = a;
            }
        }
        if (c + 1 < nb && !grid_barrier(bar, status)) return;
    }
}

// out_r[l] = sum_j M[l][j] in_r[j] over j >= l (part TRI_UPPER), j <= l
// (TRI_LOWER) or all j (FULL).
enum { TRI_UPPER = 0, TRI_LOWER = 1, FULL = 2 };
template <class T>
__global__ void __launch_bounds__(256)
k_trmv(const T *__restrict__ M, int E, int nrhs, int part, const T *__restrict__ in,
       size_t in_stride, T *__restrict__ out, size_t out_stride) {
    const int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (l >= E) return;
    const T *row = M + (size_t)l * E;
    const int jlo = part == TRI_UPPER ? l : 0, jhi = part == TRI_LOWER ? l + 1 : E;
    for (int r0 = 0; r0 < nrhs; r0 += MAXR) {
        T acc[MAXR];
#pragma unroll
        for (int r = 0; r < MAXR; ++r) acc[r] = (T)0;
        constexpr int U = 8;
        int j0 = jlo;
        for (; j0 + 32 * U <= jhi; j0 += 32 * U) {
            T v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = row[j0 + 32 * u + lane];
#pragma unroll
            for (int r = 0; r < MAXR; ++r)
                if (r0 + r < nrhs) {
                    const T *ir = in + (size_t)(r0 + r) * in_stride + j0 + lane;
#pragma unroll
                    for (int u = 0; u < U; ++u) acc[r] = fma(v[u], ir[32 * u], acc[r]);
                }
        }
        for (int j = j0 + lane; j < jhi; j += 32) {
            T v = row[j];
#pragma unroll
            for (int r = 0; r < MAXR; ++r)
                if (r0 + r < nrhs) acc[r] = fma(v, in[(size_t)(r0 + r) * in_stride + j], acc[r]);
        }
#pragma unroll
        for (int r = 0; r < MAXR; ++r) {
            if (r0 + r >= nrhs) break;
            T a = acc[r];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) out[(size_t)(r0 + r) * out_stride + l] = a;
        }
    }
}

// ---------------------------------------------------- refinement kernels ---
// w += delta (FP64 += FP32)
__global__ void k_update(double *__restrict__ w, const float *__restrict__ delta, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] += (double)delta[i];
}

// out[0] = ||a||^2, out[1] = ||b||^2 (one CTA)
__global__ void k_norms2(const double *__restrict__ a, const double *__restrict__ b, size_t n,
                         double *__restrict__ out) {
    __shared__ double red[2][32];
    double sa = 0.0, sb = 0.0;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
        sa = fma(a[i], a[i], sa);
        sb = fma(b[i], b[i], sb);
    }
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sa;
        red[1][threadIdx.x >> 5] = sb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) {
            x += red[0][wi];
            y += red[1][wi];
        }
        out[0] = x;
        out[1] = y;
    }
}

// Device-side end of a refinement without host synchronisation: the
// relative residual from out[0] = ||r||^2, out[1] = ||f||^2 into the
// workspace header, and STB_ERR_NOT_CONVERGED if it exceeds tol.
__global__ void k_refine_report(const double *__restrict__ norms, double tol, int32_t refinements,
                                int32_t *__restrict__ hdr_status, int32_t *__restrict__ hdr_refine,
                                double *__restrict__ hdr_residual) {
    const double rel = norms[1] > 0.0 ? sqrt(norms[0] / norms[1]) : sqrt(norms[0]);
    *hdr_refine = refinements;
    *hdr_residual = rel;
    if (!(rel <= tol)) atomicCAS(hdr_status, 0, STB_ERR_NOT_CONVERGED);
}

// ---------------------------------------------------------------- driver ---
// Workspace header (first 256 bytes): int32 status, int32 refinements,
// double relative residual of the last solve.
struct SolveHeader {
    int32_t status;
    int32_t refinements;
    double rel_residual;
};

struct SolveLayout {
    void *L, *Li, *LiT, *rv;  // T (L holds (V^0)^{-1} after the factorisation)
    double *hv;                   // panel right-hand sides [nrhs][PB][E]
    void *part;                   // far-history slices [nz][nrhs][PB][E] (T)
    int4 *tasks;                  // task lists of the recursive inversion of L
    float *delta;                // mixed: correction [nrhs][n_steps][E]
    double *r;                    // mixed: residual / right-hand side
    void *df;                     // mixed: scratch of the split residual product
    double *norms;                // mixed: ||r||^2, ||f||^2
    void *xf;                     // mixed, <= 8 right-hand sides: x slices of the tensor-core far history
    unsigned *bar;                // grid barrier words of the cooperative march
    int32_t *status;              // device status word of the call
    size_t bytes;
};

static SolveLayout solve_layout(int64_t E, int n_steps, int nrhs, bool mixed, void *ws, size_t cap) {
    Carve c(ws, cap);
    SolveLayout S{};
    const size_t tb = mixed ? sizeof(float) : sizeof(double);
    S.L = c.take<char>((size_t)E * E * tb);
    S.Li = c.take<char>((size_t)E * E * tb);
    S.LiT = c.take<char>((size_t)E * E * tb);
    S.rv = c.take<char>((size_t)nrhs * E * tb);
    S.hv = c.take<double>((size_t)nrhs * PB * E);
    // far-history slices: the tensor-core path of the mixed march may use more
    const int nz_max = mixed && panel_tc_supported(nrhs) ? std::max(FAR_NZ, panel_tc_max_slices())
                                                          : FAR_NZ;
    S.part = c.take<char>((size_t)nz_max * nrhs * PB * E * tb);
    S.tasks = c.take<int4>(inv_task_count((int)((E + NB - 1) / NB)));
    S.bar = c.take<unsigned>(4);
    if (mixed) {
        const size_t n = (size_t)nrhs * n_steps * E;
        S.delta = c.take<float>(n);
        S.r = c.take<double>(n);
        S.df = c.take<char>(toeplitz_split_bytes(E, n_steps, nrhs));
        S.norms = c.take<double>(2);
        if (panel_tc_supported(nrhs)) S.xf = c.take<char>(panel_tc_bytes(E, n_steps, nrhs));
    }
    S.bytes = c.off;
    return S;
}

// V^0 = L L^T, then L^{-1}, its transpose and (V^0)^{-1} = L^{-T} L^{-1}
// (written over L), all in T.
template <class AT, class T>
static stb_status factorize(const AT *V, int E, const SolveLayout &S, int32_t *status,
                            cudaStream_t s) {
    stb_status st;
    T *L = (T *)S.L, *Li = (T *)S.Li, *LiT = (T *)S.LiT;
    const size_t EE = (size_t)E * E;
    count_launch(s);
    k_copy_convert<AT, T><<<(unsigned)((EE + 255) / 256), 256, 0, s>>>(V, EE, L);
    if ((st = check_launch("k_copy_convert"))) return st;
    const int nb = (E + NB - 1) / NB;
    {  // the blocked Cholesky: one cooperative launch (4 CTAs per SM at most)
        const size_t smem = potrf_smem<T>();
        STB_CUDA(cudaFuncSetAttribute(k_potrf_coop<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        const int most = nb > 1 ? std::max(nb - 1, (nb - 1) * nb / 2) : 1;
        const int grid = std::min(most, coop_grid(k_potrf_coop<T>, 256, smem, 4));
        if (grid < 1) return fail(STB_ERR_CUDA, "factorisation: no resident grid for k_potrf_coop");
        STB_CUDA(grid_barrier_reset(S.bar, s));
        count_launch(s);
        if (cudaError_t e = launch_coop(k_potrf_coop<T>, (unsigned)grid, 256, smem, s, L, E, nb,
                                        status, S.bar)) {
            cudaGetLastError();
            return fail(STB_ERR_CUDA, "k_potrf_coop: %s", cudaGetErrorString(e));
        }
        if ((st = check_launch("k_potrf_coop"))) return st;
    }
    STB_CUDA(cudaMemsetAsync(Li, 0, EE * sizeof(T), s));
    count_launch(s);
    k_trtri_diag<T><<<nb, 64, 0, s>>>(L, Li, E);
    if ((st = check_launch("k_trtri_diag"))) return st;
    {  // off-diagonal tiles of L^{-1}: recursive halving, deepest level first
        std::vector<InvLevel> lv;
        inv_tasks(0, nb, 0, lv);  // host copy: only the counts are used
        if (!lv.empty()) {
            if ((int)lv.size() > INV_MAX_DEPTH) return fail(STB_ERR_INVALID_ARG, "E too large");
            InvOffs o{};
            int off = 0;
            for (size_t d = 0; d < lv.size(); ++d) {
                o.off[d] = off;
                o.cnt[d] = (int)lv[d].p1.size();
                off += 2 * o.cnt[d];
            }
            count_launch(s);
            k_inv_tasks<<<1, 1, 0, s>>>(nb, (int)lv.size(), o, S.tasks);
            if ((st = check_launch("k_inv_tasks"))) return st;
            T *W = LiT;  // scratch until the transpose below
            for (int d = (int)lv.size() - 1; d >= 0; --d) {
                const int4 *t1 = S.tasks + o.off[d], *t2 = t1 + o.cnt[d];
                count_launch(s);
                k_tile_gemm<T><<<(unsigned)o.cnt[d], 256, 0, s>>>(t1, L, Li, W, E, (T)1);
                if ((st = check_launch("k_tile_gemm(L21 Li11)"))) return st;
                count_launch(s);
                k_tile_gemm<T><<<(unsigned)o.cnt[d], 256, 0, s>>>(t2, Li, W, Li, E, (T)-1);
                if ((st = check_launch("k_tile_gemm(Li22 W)"))) return st;
            }
        }
    }
    count_launch(s);
    k_transpose<T><<<dim3((E + 31) / 32, (E + 31) / 32), dim3(32, 8), 0, s>>>(Li, LiT, E);
    if ((st = check_launch("k_transpose"))) return st;
    // (V^0)^{-1} = L^{-T} L^{-1} into the storage of L (no longer needed)
    count_launch(s);
    k_inverse_spd<T><<<nb * (nb + 1) / 2, 256, 0, s>>>(LiT, L, E);
    return check_launch("k_inverse_spd");
}

// March in time: x^k = L^{-T} L^{-1} (rhs^k - sum_{d>=1} V^d x^{k-d}) into x
// (T), in panels of PB steps: one far-history pass per panel (the blocks of
// the steps before the panel), then one cooperative launch for the panel's
// steps (the near history inside the panel and the product with (V^0)^{-1},
// step after step, separated by grid barriers).
template <class AT, class T>
static stb_status march(const AT *V, int E, int n_steps, int nrhs, const double *rhs, T *x,
                        const SolveLayout &S, cudaStream_t s) {
    stb_status st;
    T *rv = (T *)S.rv, *part = (T *)S.part;
    const bool vec = E % 4 == 0 && reinterpret_cast<uintptr_t>(V) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(x) % 16 == 0;
    const int rows_cta = 8 * (nrhs == 1 ? far_rows_per_warp<T, 1>() : far_rows_per_warp<T, 2>());
    const unsigned far_rows = (unsigned)((E + rows_cta - 1) / rows_cta);
    // FP32 blocks and FP32 march: the far history on the tensor cores
    constexpr bool f32 = sizeof(AT) == 4 && sizeof(T) == 4;
    const bool tc = f32 && S.xf != nullptr && panel_tc_blocks_ok((const float *)V, E);
    if (tc && (st = panel_tc_begin(E, n_steps, nrhs, S.xf, s))) return st;
    // the cooperative panel kernel: as many CTAs as row blocks, at most what
    // can be resident at once (4 per SM)
    const bool mp_vec = vec && reinterpret_cast<uintptr_t>(S.L) % 16 == 0 &&
                        reinterpret_cast<uintptr_t>(S.rv) % 16 == 0;
    int dev = 0, sms = 0;
    STB_CUDA(cudaGetDevice(&dev));
    STB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    constexpr int RW_HI = f32 ? 3 : 2;
    const bool rw3 = f32 && (E + 23) / 24 >= sms;
    const auto mp_kern =
        rw3 ? (mp_vec ? k_march_panel<AT, T, RW_HI, true> : k_march_panel<AT, T, RW_HI, false>)
            : (mp_vec ? k_march_panel<AT, T, 2, true> : k_march_panel<AT, T, 2, false>);
    const int RW = rw3 ? RW_HI : 2;
    const int mp_rows = (E + 8 * RW - 1) / (8 * RW);
    const int mp_grid = std::min(mp_rows, coop_grid(mp_kern, MP_THREADS, 0, 4));
    if (mp_grid < 1) return fail(STB_ERR_CUDA, "march: no resident grid for k_march_panel");
    STB_CUDA(grid_barrier_reset(S.bar, s));
    for (int kp = 0; kp < n_steps; kp += PB) {
        const int nb = min(PB, n_steps - kp);
        int nz = 0;
        if (kp > 0 && tc) {
            if constexpr (f32) {
                if ((st = panel_tc((const float *)V, E, n_steps, nrhs, (const float *)x, kp, nb, S.xf,
                                   (float *)part, &nz, S.status, s)))
                    return st;
            }
        } else if (kp > 0) {  // about 8 resident CTAs on each of the 152 SMs
            const int n_d = kp + nb - 1;
            nz = min(min(FAR_NZ, n_d), max(1, (int)((8 * 152 + far_rows - 1) / far_rows)));
            const int dz = (n_d + nz - 1) / nz;
            nz = (n_d + dz - 1) / dz;
            const auto kern = nrhs == 1 ? (vec ? k_history_far<AT, T, 1, true>
                                               : k_history_far<AT, T, 1, false>)
                                        : (vec ? k_history_far<AT, T, 2, true>
                                               : k_history_far<AT, T, 2, false>);
            count_launch(s);
            kern<<<dim3(far_rows, (unsigned)nz), 256, 0, s>>>(V, E, n_steps, nrhs, kp, nb, dz, x,
                                                              part);
            if ((st = check_launch("k_history_far"))) return st;
        }
        const size_t nred = (size_t)nrhs * nb * E;
        count_launch(s);
        k_far_reduce<T><<<(unsigned)((nred + 255) / 256), 256, 0, s>>>(part, nz, E, n_steps, nrhs, kp, nb,
                                                                       rhs, S.hv);
        if ((st = check_launch("k_far_reduce"))) return st;
        // the panel's steps: near history and (V^0)^{-1}, one cooperative launch
        count_launch(s);
        if (cudaError_t e = launch_coop(mp_kern, (unsigned)mp_grid, MP_THREADS, 0, s, V,
                                        (const T *)S.L, E, n_steps, nrhs, kp, nb, (const double *)S.hv,
                                        rv, x, S.bar, S.status)) {
            cudaGetLastError();
            return fail(STB_ERR_CUDA, "k_march_panel: %s", cudaGetErrorString(e));
        }
        if ((st = check_launch("k_march_panel"))) return st;
    }
    return STB_OK;
}

constexpr double REFINE_TOL = 1e-10;
constexpr int MAX_REFINE = 8;

static stb_status solve_mixed(const float *V, int E, int n_steps, int nrhs, const double *f,
                              double *w, const SolveLayout &S, int32_t *status, void *ws,
                              bool no_sync, int fixed_refine, cudaStream_t s) {
    stb_status st = factorize<float, float>(V, E, S, status, s);
    if (st) return st;
    const size_t n = (size_t)nrhs * n_steps * E;
    STB_CUDA(cudaMemsetAsync(w, 0, n * sizeof(double), s));
    const double *rhs = f;  // first pass solves with f itself
    SolveHeader hdr{STB_OK, 0, 0.0};
    const int max_refine = no_sync ? fixed_refine : MAX_REFINE;
    for (int it = 0; it <= max_refine; ++it) {
        if ((st = march<float, float>(V, E, n_steps, nrhs, rhs, S.delta, S, s))) return st;
        count_launch(s);
        k_update<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w, S.delta, n);
        if ((st = check_launch("k_update"))) return st;
        // r_it = r_{it-1} - V_h delta_it (r_{-1} = f), the product on the
        // tensor cores with split operands (about 2^-44 of the chunk scales)
        // (V's row exponents, formed by the first residual, stay in S.df)
        if ((st = toeplitz_split_f32x(V, E, n_steps, nrhs, S.delta, DF_RESIDUAL,
                                      it == 0 ? f : S.r, 0.0, S.r, S.df, status, it > 0, s)))
            return st;
        rhs = S.r;
        if (no_sync && it < max_refine) continue;  // fixed count: no norms until the end
        count_launch(s);
        k_norms2<<<1, 1024, 0, s>>>(S.r, f, n, S.norms);
        if ((st = check_launch("k_norms2"))) return st;
        if (no_sync) {
            SolveHeader *dh = static_cast<SolveHeader *>(ws);
            count_launch(s);
            k_refine_report<<<1, 1, 0, s>>>(S.norms, REFINE_TOL, it, &dh->status, &dh->refinements,
                                            &dh->rel_residual);
            return check_launch("k_refine_report");
        }
        double nrm[2];
        STB_CUDA(cudaMemcpyAsync(nrm, S.norms, sizeof nrm, cudaMemcpyDeviceToHost, s));
        STB_CUDA(cudaStreamSynchronize(s));
        hdr.refinements = it;
        hdr.rel_residual = nrm[1] > 0.0 ? std::sqrt(nrm[0] / nrm[1]) : std::sqrt(nrm[0]);
        if (hdr.rel_residual <= REFINE_TOL || !std::isfinite(hdr.rel_residual)) break;
    }
    int32_t dev_status = 0;
    STB_CUDA(cudaMemcpyAsync(&dev_status, status, sizeof dev_status, cudaMemcpyDeviceToHost, s));
    STB_CUDA(cudaStreamSynchronize(s));
    hdr.status = dev_status;
    if (dev_status == STB_OK && !(hdr.rel_residual <= REFINE_TOL)) hdr.status = STB_ERR_NOT_CONVERGED;
    STB_CUDA(cudaMemcpyAsync(ws, &hdr, sizeof hdr, cudaMemcpyHostToDevice, s));
    STB_CUDA(cudaStreamSynchronize(s));
    return STB_OK;
}

// ---------------------------------------------- dense SPD helpers ---
// The factorisation and explicit inverse above, for any SPD FP64 matrix (the
// piecewise-linear mass matrix of the L2 projection, Sec. 3.4).
size_t spd_inverse_bytes(int64_t n) {
    return align256(solve_layout(n, 1, 1, false, nullptr, 0).bytes);
}

stb_status spd_inverse(const double *M, int64_t n, void *scratch, size_t cap, int32_t *status,
                       double **inv, cudaStream_t s) {
    if (n < 1 || n > 65535) return fail(STB_ERR_INVALID_ARG, "SPD inverse needs 1 <= n <= 65535");
    SolveLayout S = solve_layout(n, 1, 1, false, scratch, cap);
    if (!scratch || S.bytes > cap) return fail(STB_ERR_INVALID_ARG, "SPD inverse scratch too small");
    *inv = (double *)S.L;
    return factorize<double, double>(M, (int)n, S, status, s);
}

// out_v = A in_v for nvec vectors of length n (A row-major n x n)
stb_status dense_apply(const double *A, int64_t n, int64_t nvec, const double *in, double *out,
                       cudaStream_t s) {
    if (n < 1 || n > 65535 || nvec < 1 || nvec > INT32_MAX)
        return fail(STB_ERR_INVALID_ARG, "bad dense product size");
    count_launch(s);
    k_trmv<double><<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(A, (int)n, (int)nvec, FULL, in,
                                                                   (size_t)n, out, (size_t)n);
    return check_launch("k_trmv");
}

}  // namespace stb

using namespace stb;

// The forward-substitution solve for blocks of size E x E (E triangles for
// V_h w = f, E nodes for D_h u = f).
static stb_status solve_size(int64_t E, const stb_params *p, int32_t nrhs, size_t *bytes) {
    if (!p || !bytes || nrhs < 1 || p->n_steps < 1)
        return fail(STB_ERR_INVALID_ARG, "invalid argument");
    const bool mixed = p->precision == STB_PREC_MIXED;
    *bytes = align256(solve_layout(E, p->n_steps, nrhs, mixed, nullptr, 0).bytes);
    return STB_OK;
}

static stb_status solve_blocks(int64_t E, const stb_params *p, const void *V, const double *f,
                               int32_t nrhs, double *w, void *ws, size_t ws_bytes,
                               stb_stream stream);

// ------------------------------------------------- grid barrier self test ---
// Every CTA but `skip` (-1: none) enters one grid barrier with the given
// limit; out[b] = 1 if CTA b passed it, 0 if its wait gave up, 2 if it
// skipped.  With a CTA skipping, the others' waits expire: STB_ERR_TIMEOUT.
__global__ void k_selftest_grid(unsigned *bar, int32_t *status, int skip, uint64_t limit_ns,
                                int32_t *out) {
    int32_t r = 2;
    if ((int)blockIdx.x != skip) r = grid_barrier(bar, status, limit_ns) ? 1 : 0;
    if (threadIdx.x == 0) out[blockIdx.x] = r;
}

extern "C" stb_status stb_selftest_grid_barrier(int32_t n_cta, int32_t skip, int64_t limit_ns,
                                                void *ws, size_t ws_bytes, stb_stream stream) {
    if (n_cta < 1 || skip < -1 || skip >= n_cta)
        return fail(STB_ERR_INVALID_ARG, "need n_cta >= 1 and -1 <= skip < n_cta");
    if (limit_ns < 1000 || limit_ns > 10000000000ll)
        return fail(STB_ERR_INVALID_ARG, "limit_ns must lie in [1000, 1e10]");
    const int most = coop_grid(k_selftest_grid, 128, 0, 1);
    if (n_cta > most) return fail(STB_ERR_INVALID_ARG, "n_cta above one CTA per SM (%d)", most);
    const size_t need = 256 + 256 + (size_t)n_cta * sizeof(int32_t);
    stb_status st = check_workspace(ws, ws_bytes, need);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 512, s));
    unsigned *bar = reinterpret_cast<unsigned *>(static_cast<char *>(ws) + 256);
    int32_t *out = reinterpret_cast<int32_t *>(static_cast<char *>(ws) + 512);
    count_launch(s);
    if (cudaError_t e = launch_coop(k_selftest_grid, (unsigned)n_cta, 128, 0, s, bar, status_word(ws),
                                    (int)skip, (uint64_t)limit_ns, out)) {
        cudaGetLastError();
        return fail(STB_ERR_CUDA, "k_selftest_grid: %s", cudaGetErrorString(e));
    }
    return check_launch("k_selftest_grid");
}

extern "C" stb_status stb_solve_workspace_size(const stb_mesh *mesh, const stb_params *p,
                                               int32_t nrhs, size_t *bytes) {
    if (!mesh) return fail(STB_ERR_INVALID_ARG, "invalid argument");
    return solve_size(mesh->m.n_tris, p, nrhs, bytes);
}

extern "C" stb_status stb_dirichlet_solve(const stb_mesh *mesh, const stb_params *p, const void *V,
                                          const double *f, int32_t nrhs, double *w, void *ws,
                                          size_t ws_bytes, stb_stream stream) {
    if (!mesh) return fail(STB_ERR_INVALID_ARG, "null argument");
    return solve_blocks(mesh->m.n_tris, p, V, f, nrhs, w, ws, ws_bytes, stream);
}

extern "C" stb_status stb_neumann_solve_workspace_size(const stb_mesh *mesh, const stb_params *p,
                                                       int32_t nrhs, size_t *bytes) {
    if (!mesh) return fail(STB_ERR_INVALID_ARG, "invalid argument");
    return solve_size(mesh->m.n_nodes, p, nrhs, bytes);
}

extern "C" stb_status stb_neumann_solve(const stb_mesh *mesh, const stb_params *p, const void *D,
                                        const double *f, int32_t nrhs, double *u, void *ws,
                                        size_t ws_bytes, stb_stream stream) {
    if (!mesh) return fail(STB_ERR_INVALID_ARG, "null argument");
    return solve_blocks(mesh->m.n_nodes, p, D, f, nrhs, u, ws, ws_bytes, stream);
}

static stb_status solve_blocks(int64_t E, const stb_params *p, const void *V, const double *f,
                               int32_t nrhs, double *w, void *ws, size_t ws_bytes,
                               stb_stream stream) {
    if (!p || !V || !f || !w || nrhs < 1) return fail(STB_ERR_INVALID_ARG, "null argument");
    if (p->n_steps < 1) return fail(STB_ERR_INVALID_ARG, "n_steps must be >= 1");
    if (p->storage != STB_STORE_F64 && p->storage != STB_STORE_F32)
        return fail(STB_ERR_INVALID_ARG, "bad storage");
    const bool mixed = p->precision == STB_PREC_MIXED;
    if (mixed && p->storage != STB_STORE_F32)
        return fail(STB_ERR_INVALID_ARG, "mixed-precision solve needs STB_STORE_F32 blocks");
    if (E > 65535) return fail(STB_ERR_INVALID_ARG, "E must be <= 65535");
    SolveLayout S = solve_layout(E, p->n_steps, nrhs, mixed, ws, ws_bytes);
    stb_status st = check_workspace(ws, ws_bytes, S.bytes);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    int32_t *status = status_word(ws);
    S.status = status;
    if (mixed) {
        st = solve_mixed((const float *)V, (int)E, p->n_steps, nrhs, f, w, S, status, ws,
                         (p->flags & STB_FLAG_NO_SYNC) != 0,
                         std::max(1, (p->flags >> 8) & 15), s);
        if (st) return st;
    } else {
        if (p->storage == STB_STORE_F64) {
            st = factorize<double, double>((const double *)V, (int)E, S, status, s);
            if (!st) st = march<double, double>((const double *)V, (int)E, p->n_steps, nrhs, f, w, S, s);
        } else {
            st = factorize<float, double>((const float *)V, (int)E, S, status, s);
            if (!st) st = march<float, double>((const float *)V, (int)E, p->n_steps, nrhs, f, w, S, s);
        }
        if (st) return st;
    }
    if (p->flags & STB_FLAG_NO_SYNC) return STB_OK;  // status stays in the workspace
    return stb_workspace_status(ws, stream);
}

extern "C" stb_status stb_solve_report(const void *ws, stb_stream stream, int32_t *refinements,
                                       double *rel_residual) {
    if (!ws) return fail(STB_ERR_INVALID_ARG, "workspace is NULL");
    SolveHeader hdr{};
    STB_CUDA(cudaMemcpyAsync(&hdr, ws, sizeof hdr, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    STB_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (refinements) *refinements = hdr.refinements;
    if (rel_residual) *rel_residual = hdr.rel_residual;
    return STB_OK;
}
