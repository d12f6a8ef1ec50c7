// stb_solve.cu -- solution of the block lower-triangular Toeplitz system
// V_h w = f of the Dirichlet problem (eq. V_mat, Sec. 3.4) by block forward
// substitution in time:
//     w^k = (V^0)^{-1} ( f^k - sum_{d=1}^{k} V^d w^{k-d} ),  k = 0..E_t-1.
// V^0 is symmetric positive definite; it is factorised once, V^0 = L L^T, by
// a right-looking blocked Cholesky (64 x 64 tiles), L is inverted blockwise,
// and every time step is then three matrix-vector kernels: the history sum
// (reads V^1..V^k once, all right-hand sides together), z = L^{-1} r and
// w^k = L^{-T} z.  All FP64.
#include <cmath>

#include "stb_internal.h"

namespace stb {

constexpr int NB = 64;

template <class AT>
__global__ void k_copy_to_f64(const AT *__restrict__ src, size_t n, double *__restrict__ dst) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (double)src[i];
}

// Cholesky of diagonal tile kb (updates from the left already applied).
__global__ void __launch_bounds__(256) k_potrf_diag(double *__restrict__ L, int E, int kb,
                                                    int32_t *__restrict__ status) {
    __shared__ double T[NB][NB + 1];
    const int b0 = kb * NB, n = min(NB, E - b0);
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
        int i = t / NB, j = t % NB;
        T[i][j] = (i < n && j < n && j <= i) ? L[(size_t)(b0 + i) * E + b0 + j] : 0.0;
    }
    __syncthreads();
    for (int c = 0; c < n; ++c) {
        if (threadIdx.x == 0) {
            double p = T[c][c];
            if (!(p > 0.0)) {
                atomicCAS(status, 0, STB_ERR_NOT_SPD);
                p = 1.0;
            }
            T[c][c] = sqrt(p);
        }
        __syncthreads();
        const double inv = 1.0 / T[c][c];
        for (int i = c + 1 + threadIdx.x; i < n; i += blockDim.x) T[i][c] *= inv;
        __syncthreads();
        const int m = n - c - 1;  // trailing size
        for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
            int i = c + 1 + t / m, j = c + 1 + t % m;
            if (j <= i) T[i][j] = fma(-T[i][c], T[j][c], T[i][j]);
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        int i = t / n, j = t % n;
        L[(size_t)(b0 + i) * E + b0 + j] = j <= i ? T[i][j] : 0.0;
    }
}

// Panel: L_ik = A_ik L_kk^{-T} for the tile rows i > kb.
__global__ void __launch_bounds__(128) k_trsm_panel(double *__restrict__ L, int E, int kb) {
    __shared__ double Lk[NB][NB + 1];
    __shared__ double A[NB][NB + 1];
    const int b0 = kb * NB, n = min(NB, E - b0);
    const int i0 = (kb + 1 + blockIdx.x) * NB, mrows = min(NB, E - i0);
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
        int i = t / NB, j = t % NB;
        Lk[i][j] = (i < n && j < n) ? L[(size_t)(b0 + i) * E + b0 + j] : 0.0;
        A[i][j] = (i < mrows && j < n) ? L[(size_t)(i0 + i) * E + b0 + j] : 0.0;
    }
    __syncthreads();
    for (int row = threadIdx.x; row < mrows; row += blockDim.x) {
        for (int c = 0; c < n; ++c) {
            double x = A[row][c];
            for (int cc = 0; cc < c; ++cc) x = fma(-A[row][cc], Lk[c][cc], x);
            A[row][c] = x / Lk[c][c];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < mrows * n; t += blockDim.x) {
        int i = t / n, j = t % n;
        L[(size_t)(i0 + i) * E + b0 + j] = A[i][j];
    }
}

// 64x64 FP64 tile product helper: acc (4x4 per thread, 256 threads) +=
// P (rows of tile) * Q^T, both read from global in 32-wide chunks.
struct TileAcc {
    double v[4][4];
};

__device__ __forceinline__ void tile_mma_abt(TileAcc &acc, const double *P, size_t ldp, int prow,
                                             int pcol, const double *Q, size_t ldq, int qrow,
                                             int qcol, int E, int kn, double (*Ps)[33],
                                             double (*Qs)[33]) {
    // acc[i][j] += sum_k P[prow+i][pcol+k] * Q[qrow+j][qcol+k], k < kn
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    for (int k0 = 0; k0 < kn; k0 += 32) {
        for (int t = threadIdx.x; t < NB * 32; t += blockDim.x) {
            int r = t / 32, kk = t % 32;
            int pr = prow + r, qr = qrow + r, pc = pcol + k0 + kk, qc = qcol + k0 + kk;
            Ps[r][kk] = (pr < E && k0 + kk < kn) ? P[(size_t)pr * ldp + pc] : 0.0;
            Qs[r][kk] = (qr < E && k0 + kk < kn) ? Q[(size_t)qr * ldq + qc] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 32; ++kk) {
            double a[4], b[4];
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

// Trailing update A_ij -= L_ik L_jk^T for kb < j <= i.
__global__ void __launch_bounds__(256) k_syrk_update(double *__restrict__ L, int E, int kb, int nb) {
    __shared__ double Ps[NB][33], Qs[NB][33];
    const int t = blockIdx.x;
    int ii = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
    while (ii * (ii + 1) / 2 > t) --ii;
    const int jj = t - ii * (ii + 1) / 2;
    const int i0 = (kb + 1 + ii) * NB, j0 = (kb + 1 + jj) * NB, b0 = kb * NB;
    const int kn = min(NB, E - b0);
    TileAcc acc;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc.v[u][v] = 0.0;
    tile_mma_abt(acc, L, E, i0, b0, L, E, j0, b0, E, kn, Ps, Qs);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    for (int u = 0; u < 4; ++u)
        for (int v = 0; v < 4; ++v) {
            int r = i0 + 4 * ty + u, c = j0 + 4 * tx + v;
            if (r < E && c < E) L[(size_t)r * E + c] -= acc.v[u][v];
        }
    (void)nb;
}

// Inverse of every diagonal tile of L (lower triangular), in parallel.
__global__ void __launch_bounds__(64) k_trtri_diag(const double *__restrict__ L,
                                                   double *__restrict__ Li, int E) {
    __shared__ double T[NB][NB + 1];
    __shared__ double X[NB][NB + 1];
    const int b0 = blockIdx.x * NB, n = min(NB, E - b0);
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
        int i = t / NB, j = t % NB;
        T[i][j] = (i < n && j < n) ? L[(size_t)(b0 + i) * E + b0 + j] : 0.0;
        X[i][j] = 0.0;
    }
    __syncthreads();
    const int c = threadIdx.x;  // column of the inverse
    if (c < n) {
        for (int i = c; i < n; ++i) {
            double x = (i == c) ? 1.0 : 0.0;
            for (int m = c; m < i; ++m) x = fma(-T[i][m], X[m][c], x);
            X[i][c] = x / T[i][i];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        int i = t / n, j = t % n;
        Li[(size_t)(b0 + i) * E + b0 + j] = X[i][j];
    }
}

// Tile row i of L^{-1}: Li_ij = -Li_ii sum_{m=j}^{i-1} L_im Li_mj, j < i.
// Li tiles are read transposed through a staging copy (Q^T form).
__global__ void __launch_bounds__(256) k_trtri_row(const double *__restrict__ L,
                                                   double *__restrict__ Li, int E, int i) {
    __shared__ double Ps[NB][33], Qs[NB][33];
    __shared__ double Tt[NB][NB + 1];  // T^T, T = sum L_im Li_mj
    const int j = blockIdx.x;
    const int i0 = i * NB, j0 = j * NB;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    TileAcc acc;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc.v[u][v] = 0.0;
    for (int m = j; m < i; ++m) {
        const int m0 = m * NB;
        // acc[r][c] += sum_k L[i0+r][m0+k] * Li[m0+k][j0+c]  (Q = Li^T: Q[c][k] = Li[m0+k][j0+c])
        for (int k0 = 0; k0 < NB; k0 += 32) {
            for (int t = threadIdx.x; t < NB * 32; t += blockDim.x) {
                int r = t / 32, kk = t % 32;
                int gr = i0 + r, gk = m0 + k0 + kk, gc = j0 + r;
                Ps[r][kk] = (gr < E && gk < E) ? L[(size_t)gr * E + gk] : 0.0;
                Qs[r][kk] = (gk < E && gc < E) ? Li[(size_t)gk * E + gc] : 0.0;
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < 32; ++kk) {
                double a[4], b[4];
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
    // store T^T so that the second product reads it as Q[c][k] = T[k][c]
    for (int u = 0; u < 4; ++u)
        for (int v = 0; v < 4; ++v) Tt[4 * tx + v][4 * ty + u] = acc.v[u][v];
    __syncthreads();
    TileAcc out;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) out.v[u][v] = 0.0;
    for (int k0 = 0; k0 < NB; k0 += 32) {
        for (int t = threadIdx.x; t < NB * 32; t += blockDim.x) {
            int r = t / 32, kk = t % 32;
            int gr = i0 + r, gk = i0 + k0 + kk;
            Ps[r][kk] = (gr < E && gk < E) ? Li[(size_t)gr * E + gk] : 0.0;
            Qs[r][kk] = Tt[r][k0 + kk];
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 32; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = Ps[4 * ty + u][kk];
                b[u] = Qs[4 * tx + u][kk];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) out.v[u][v] = fma(a[u], b[v], out.v[u][v]);
        }
        __syncthreads();
    }
    for (int u = 0; u < 4; ++u)
        for (int v = 0; v < 4; ++v) {
            int r = i0 + 4 * ty + u, c = j0 + 4 * tx + v;
            if (r < E && c < E) Li[(size_t)r * E + c] = -out.v[u][v];
        }
}

__global__ void k_transpose(const double *__restrict__ A, double *__restrict__ B, int E) {
    __shared__ double t[32][33];
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

// r_r = f_r^k - sum_{d=1}^{k} V^d w_r^{k-d}: one warp per row l, all rhs of
// the group [r0, r0 + nr) together so that each V^d row is read once.
template <class AT>
__global__ void __launch_bounds__(256)
k_history(const AT *__restrict__ V, int E, int n_steps, int r0, int nr, int k,
          const double *__restrict__ f, const double *__restrict__ w, double *__restrict__ rv) {
    const int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (l >= E) return;
    double acc[MAXR];
#pragma unroll
    for (int r = 0; r < MAXR; ++r) acc[r] = 0.0;
    const size_t EE = (size_t)E * E, SE = (size_t)n_steps * E;
    constexpr int U = 8;  // independent loads in flight per lane
    for (int d = 1; d <= k; ++d) {
        const AT *row = V + d * EE + (size_t)l * E;
        const double *wk = w + (size_t)(k - d) * E;
        int j0 = 0;
        for (; j0 + 32 * U <= E; j0 += 32 * U) {
            double v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = (double)row[j0 + 32 * u + lane];
#pragma unroll
            for (int r = 0; r < MAXR; ++r)
                if (r < nr) {
                    const double *wr = wk + (size_t)(r0 + r) * SE + j0 + lane;
#pragma unroll
                    for (int u = 0; u < U; ++u) acc[r] = fma(v[u], wr[32 * u], acc[r]);
                }
        }
        for (int j = j0 + lane; j < E; j += 32) {
            double v = (double)row[j];
#pragma unroll
            for (int r = 0; r < MAXR; ++r)
                if (r < nr) acc[r] = fma(v, wk[(size_t)(r0 + r) * SE + j], acc[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
        if (r >= nr) break;
        double a = acc[r];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) rv[(size_t)(r0 + r) * E + l] = f[(size_t)(r0 + r) * SE + (size_t)k * E + l] - a;
    }
}

// out_r[l] = sum_{j in tri(l)} M[l][j] in_r[j]; lower: j <= l, else j >= l.
__global__ void __launch_bounds__(256)
k_trmv(const double *__restrict__ M, int E, int nrhs, int lower, const double *__restrict__ in,
       size_t in_stride, double *__restrict__ out, size_t out_stride) {
    const int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (l >= E) return;
    const double *row = M + (size_t)l * E;
    const int jlo = lower ? 0 : l, jhi = lower ? l + 1 : E;
    for (int r0 = 0; r0 < nrhs; r0 += MAXR) {
        double acc[MAXR];
#pragma unroll
        for (int r = 0; r < MAXR; ++r) acc[r] = 0.0;
        constexpr int U = 8;
        int j0 = jlo;
        for (; j0 + 32 * U <= jhi; j0 += 32 * U) {
            double v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = row[j0 + 32 * u + lane];
#pragma unroll
            for (int r = 0; r < MAXR; ++r)
                if (r0 + r < nrhs) {
                    const double *ir = in + (size_t)(r0 + r) * in_stride + j0 + lane;
#pragma unroll
                    for (int u = 0; u < U; ++u) acc[r] = fma(v[u], ir[32 * u], acc[r]);
                }
        }
        for (int j = j0 + lane; j < jhi; j += 32) {
            double v = row[j];
#pragma unroll
            for (int r = 0; r < MAXR; ++r)
                if (r0 + r < nrhs) acc[r] = fma(v, in[(size_t)(r0 + r) * in_stride + j], acc[r]);
        }
#pragma unroll
        for (int r = 0; r < MAXR; ++r) {
            if (r0 + r >= nrhs) break;
            double a = acc[r];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) out[(size_t)(r0 + r) * out_stride + l] = a;
        }
    }
}

struct SolveLayout {
    double *L, *Li, *LiT, *rv, *zv;
    size_t bytes;
};

static SolveLayout solve_layout(int64_t E, int nrhs, void *ws, size_t cap) {
    Carve c(ws, cap);
    SolveLayout S{};
    S.L = c.take<double>((size_t)E * E);
    S.Li = c.take<double>((size_t)E * E);
    S.LiT = c.take<double>((size_t)E * E);
    S.rv = c.take<double>((size_t)nrhs * E);
    S.zv = c.take<double>((size_t)nrhs * E);
    S.bytes = c.off;
    return S;
}

template <class AT>
static stb_status run_solve(const AT *V, int E, int n_steps, int nrhs, const double *f, double *w,
                            const SolveLayout &S, int32_t *status, cudaStream_t s) {
    stb_status st;
    const size_t EE = (size_t)E * E;
    count_launch(s);
    k_copy_to_f64<AT><<<(unsigned)((EE + 255) / 256), 256, 0, s>>>(V, EE, S.L);
    if ((st = check_launch("k_copy_to_f64"))) return st;
    const int nb = (E + NB - 1) / NB;
    for (int kb = 0; kb < nb; ++kb) {
        count_launch(s);
        k_potrf_diag<<<1, 256, 0, s>>>(S.L, E, kb, status);
        if ((st = check_launch("k_potrf_diag"))) return st;
        const int m = nb - kb - 1;
        if (m == 0) break;
        count_launch(s);
        k_trsm_panel<<<m, 128, 0, s>>>(S.L, E, kb);
        if ((st = check_launch("k_trsm_panel"))) return st;
        count_launch(s);
        k_syrk_update<<<m * (m + 1) / 2, 256, 0, s>>>(S.L, E, kb, nb);
        if ((st = check_launch("k_syrk_update"))) return st;
    }
    STB_CUDA(cudaMemsetAsync(S.Li, 0, EE * sizeof(double), s));
    count_launch(s);
    k_trtri_diag<<<nb, 64, 0, s>>>(S.L, S.Li, E);
    if ((st = check_launch("k_trtri_diag"))) return st;
    for (int i = 1; i < nb; ++i) {
        count_launch(s);
        k_trtri_row<<<i, 256, 0, s>>>(S.L, S.Li, E, i);
        if ((st = check_launch("k_trtri_row"))) return st;
    }
    count_launch(s);
    k_transpose<<<dim3((E + 31) / 32, (E + 31) / 32), dim3(32, 8), 0, s>>>(S.Li, S.LiT, E);
    if ((st = check_launch("k_transpose"))) return st;
    const unsigned rows_blocks = (unsigned)((E * 32 + 255) / 256);
    const size_t SE = (size_t)n_steps * E;
    for (int k = 0; k < n_steps; ++k) {
        for (int r0 = 0; r0 < nrhs; r0 += MAXR) {
            count_launch(s);
            k_history<AT><<<rows_blocks, 256, 0, s>>>(V, E, n_steps, r0, min(MAXR, nrhs - r0), k, f,
                                                      w, S.rv);
            if ((st = check_launch("k_history"))) return st;
        }
        count_launch(s);
        k_trmv<<<rows_blocks, 256, 0, s>>>(S.Li, E, nrhs, 1, S.rv, E, S.zv, E);
        if ((st = check_launch("k_trmv(L^-1)"))) return st;
        count_launch(s);
        k_trmv<<<rows_blocks, 256, 0, s>>>(S.LiT, E, nrhs, 0, S.zv, E, w + (size_t)k * E, SE);
        if ((st = check_launch("k_trmv(L^-T)"))) return st;
    }
    return STB_OK;
}

}  // namespace stb

using namespace stb;

extern "C" stb_status stb_solve_workspace_size(const stb_mesh *mesh, const stb_params *p,
                                               int32_t nrhs, size_t *bytes) {
    if (!mesh || !p || !bytes || nrhs < 1) return fail(STB_ERR_INVALID_ARG, "invalid argument");
    *bytes = align256(solve_layout(mesh->m.n_tris, nrhs, nullptr, 0).bytes);
    return STB_OK;
}

extern "C" stb_status stb_dirichlet_solve(const stb_mesh *mesh, const stb_params *p, const void *V,
                                          const double *f, int32_t nrhs, double *w, void *ws,
                                          size_t ws_bytes, stb_stream stream) {
    if (!mesh || !p || !V || !f || !w || nrhs < 1) return fail(STB_ERR_INVALID_ARG, "null argument");
    if (p->n_steps < 1) return fail(STB_ERR_INVALID_ARG, "n_steps must be >= 1");
    if (p->storage != STB_STORE_F64 && p->storage != STB_STORE_F32)
        return fail(STB_ERR_INVALID_ARG, "bad storage");
    const int64_t E = mesh->m.n_tris;
    if (E > 65535) return fail(STB_ERR_INVALID_ARG, "E must be <= 65535");
    SolveLayout S = solve_layout(E, nrhs, ws, ws_bytes);
    stb_status st = check_workspace(ws, ws_bytes, S.bytes);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    int32_t *status = status_word(ws);
    if (p->storage == STB_STORE_F64)
        st = run_solve<double>((const double *)V, (int)E, p->n_steps, nrhs, f, w, S, status, s);
    else
        st = run_solve<float>((const float *)V, (int)E, p->n_steps, nrhs, f, w, S, status, s);
    if (st) return st;
    return stb_workspace_status(ws, stream);
}
