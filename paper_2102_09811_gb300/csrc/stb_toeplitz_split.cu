// stb_toeplitz_split.cu -- block-Toeplitz product (eq. V_mat) of FP32 blocks
// with an FP64 (or FP32) vector on the tcgen05 tensor cores, with about 44
// bits of accuracy relative to the magnitudes of 64-column chunks:
//
//   y_r^k = beta y_r^k + sum_{d=0}^{k} A^d x_r^{k-d}     (or y = f - that sum)
//
// Split operands with exact accumulation (the error-free splitting idea of
// Ozaki, Ogita and Oishi).  For each row l, block d and chunk of SP_RC = 64
// columns j, the row segment is scaled by 2^-e, 2^e the power of two just
// above its largest magnitude, and cut into five bf16 slices; slice i holds
// integer digits D_i of weight 2^(-8-9i), |D_i| <= 256 (balanced, round to
// nearest: 44 bits of the scaled segment).  The same is done for x per
// (step, right-hand side, chunk) with 2^g.  A product of two digits is an
// integer of at most 16 bits, so the sum of all slice products of one level
// s = i + j over a chunk, at most (s+1) 64 2^16 <= 2^24 units of
// 2^(-16-9s) for s <= 3, is exact in the FP32 accumulator of the tensor
// core, whatever its rounding.  Products with s <= 4 are formed (15 per
// chunk), levels 0, 1, 2 and 3 in their own accumulators, level 4 added into
// level 3 (its rounding there stays near 2^-45 of the chunk scale).  After
// every chunk the four accumulators are read back, combined exactly into a
// float pair, scaled by 2^(e+g) and added to a double-float running sum per
// (row, column); the partial sums of the CTAs are added in FP64.  The error
// is bounded per chunk, relative to the chunk maxima of |A| and |x| (not to
// |A||x| entrywise), and does not grow with the length of the sum.  (With
// SP_RC = 128 the first digits are held to 128 so that levels 0..2 stay
// exact over 128 terms; that variant reads back half as often but keeps 43
// bits.)
//
// Layout.  Right-hand sides are padded to rpad (a power of two <= 64) and a
// box of 64 output columns is S = 64 / rpad steps x rpad right-hand sides,
// column q = (k - n0) * rpad + r.  The x slices are stored step-major with S
// zero steps in front and 64 zero rows behind, Xs[i][(S + m) rpad + r][j]
// (bf16, j padded to a multiple of SP_RC), so that the B tile of (block d, box
// n0, 64-column piece, slice i) is the contiguous 64-row window starting at
// row (S + n0 - d) rpad: one 2-D TMA box (128-byte swizzle).  The A slices are
// formed in shared memory by the CTA itself from the FP32 blocks (read once
// per box from HBM), written in the same swizzled layout the MMA descriptor
// expects; the row exponents e come from a pre-pass over A.
//
// CTA = 128 rows x one box x a range of blocks d; 18 warps:
//   warp 0: TMA producer of the x slices (2-stage ring of 5 tiles),
//   warp 1: tensor-memory allocation (512 columns: 2 buffers x 4 levels x 64)
//   and MMA issuer (kind::f16, bf16 operands, M = 128, K = 16; A slice i
//   meets x slices 0 .. 3-i in one MMA of N = 64 (4 - i), the levels i .. 3
//   being adjacent accumulators, and x slice 4-i in one of N = 64: nine MMAs
//   per 16 columns instead of fifteen, fewer re-reads of the A tile),
//   warps 2..9: slicers -- each thread loads 32 columns of one row of the
//   next 64-column piece of A (prefetched into L2) and forms their five
//   slices into a 7-slot ring,
//   warps 10..17: read-back -- each thread owns one tile row (TMEM lane) and
//   32 output columns and adds every chunk's four accumulators to its
//   running sums (high parts in registers, low parts in shared memory).
// The row exponents come from a pre-pass over A, so the two worker roles
// share no data and overlap freely.
// Every mbarrier wait is bounded (2 s); an expired wait sets STB_ERR_TIMEOUT in
// the status word and the CTA winds down without hanging.
#include <cuda_bf16.h>

#include <algorithm>

#include "stb_tc.cuh"
#include "stb_toeplitz.h"

namespace stb {

constexpr int SP_M = 128;       // rows per CTA (MMA M)
constexpr int SP_N = 64;        // output columns per box (MMA N)
constexpr int SP_KC = 64;       // columns j per piece (one 128-byte swizzled row of bf16)
constexpr int SP_RC = 64;       // columns j per scale chunk / read-back (64 or 128)
constexpr int SP_PPC = SP_RC / SP_KC;  // pieces per chunk
// extra scale bit: with 128-column chunks the first digits stay within 128 so
// that level 2 is exact over 128 terms; with 64 columns they may reach 256
constexpr int SP_E1 = SP_PPC == 2 ? 1 : 0;
constexpr int SP_NS = 5;        // slices per operand
constexpr int SP_NL = 4;        // accumulators per buffer (levels 0, 1, 2, 3+4)
constexpr int SP_SLICERS = 256;   // 8 slicer warps: 32 columns j of one row each
constexpr int SP_READERS = 256;   // 8 read-back warps: 2 per TMEM lane quarter, 32 columns each
constexpr int SP_WORKERS = SP_SLICERS + SP_READERS;
constexpr int SP_THREADS = 64 + SP_WORKERS;
constexpr uint32_t SP_A_BYTES = SP_M * SP_KC * 2;          // 16 KB
constexpr uint32_t SP_B_BYTES = SP_N * SP_KC * 2;          // 8 KB per slice
constexpr uint32_t SP_BSTAGE = SP_NS * SP_B_BYTES;         // 40 KB
constexpr uint32_t SP_TMEM_COLS = 2 * SP_NL * SP_N;  // 512
constexpr uint32_t SP_IDESC = idesc_bf16(SP_M, SP_N);
// Shared memory.  TA (E a multiple of 4, A 16-byte aligned): the FP32 A tile
// of a piece arrives by TMA (two 32-column halves, 128-byte swizzle) in one
// stage and the slicers read it from there; otherwise they load their row
// segments themselves and the A-slice ring has two more slots.
template <bool TA>
struct SplitShape {
    static constexpr int NA = TA ? 5 : 7;  // A-slice slots
    static constexpr int NF = TA ? 1 : 0;  // FP32 A stages
    static constexpr uint32_t F_HALF = SP_M * 128, F_BYTES = 2 * F_HALF;
    static constexpr uint32_t OFF_F = NA * SP_A_BYTES;
    static constexpr uint32_t OFF_B = OFF_F + NF * F_BYTES;
    // low parts of the read-back's running sums, float2 [32 column pairs][128 rows]
    static constexpr uint32_t OFF_AL = OFF_B + 2 * SP_BSTAGE;
    static constexpr uint32_t OFF_BAR = OFF_AL + (SP_N / 2) * SP_M * 8;
    // barriers: bfull[2] bempty[2] afull[NA] aempty[NA] accfull[2] accempty[2]
    // drain ffull[NF] fempty[NF]
    static constexpr int NBAR = 2 + 2 + NA + NA + 2 + 2 + 1 + 2 * NF;
    static constexpr uint32_t OFF_MISC = OFF_BAR + NBAR * 8;
    static constexpr size_t SMEM = OFF_MISC + 16 + 1024;  // + alignment slack
    static_assert(SMEM <= 232448, "shared memory of the split product");
};

__device__ __forceinline__ float pow2f(int k) {  // 2^k; 0 below 2^-149, +inf above 2^127
    if (k >= -126) return __int_as_float(min(k + 127, 255) << 23);
    if (k >= -149) return __int_as_float(1 << (k + 149));
    return 0.f;
}
// the smallest e with 2^e > m for a finite m >= 0 (-126 for m = 0 or subnormal)
__device__ __forceinline__ int scale_exp(float m) {
    const int ex = (__float_as_int(m) >> 23) & 0xff;
    return ex == 0 ? -126 : ex - 126;
}
__device__ __forceinline__ float2 sub2(float2 u, float2 v) {  // u - v, one rounding
    return __ffma2_rn(v, make_float2(-1.f, -1.f), u);
}

// ------------------------------------------------------ x slices (step-major)
// Xs[i][R][j] for R = (S + m) rpad + r, bf16; xsc[c][R] = 2^(g+1) of the
// 128-column chunk c (0 for the padding rows).  One warp per (R, chunk),
// four values per lane.
template <class XT>
__global__ void k_split_x(const XT *__restrict__ x, int E, int E_pad, int n_steps, int nrhs,
                          int rpad, int S, int rowsX, int n_rc, __nv_bfloat16 *__restrict__ Xs,
                          float *__restrict__ xsc) {
    const size_t wid = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (size_t)rowsX * n_rc) return;
    const int R = (int)(wid % rowsX), c = (int)(wid / rowsX);
    const int m = R / rpad - S, r = R % rpad;
    const int j0 = c * SP_RC + 2 * lane;  // lane's pairs at j0 (and j0 + 64)
    constexpr int NV = SP_RC / 32;
    double v[NV];
#pragma unroll
    for (int u = 0; u < NV; ++u) v[u] = 0.0;
    if (m >= 0 && m < n_steps && r < nrhs) {
        const XT *xr = x + ((size_t)r * n_steps + m) * E;
#pragma unroll
        for (int u = 0; u < NV; ++u) {
            const int j = j0 + (u >> 1) * SP_KC + (u & 1);
            if (j < E) v[u] = (double)xr[j];
        }
    }
    double mx = 0.0;
#pragma unroll
    for (int u = 0; u < NV; ++u) mx = fmax(mx, fabs(v[u]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    // g: the smallest power of two above the chunk maximum (0 for a zero chunk);
    // the segment is scaled by 2^-(g+1) so that |first digit| <= 128
    const int ex = (int)((__double_as_longlong(mx) >> 52) & 0x7ff);
    const int g = mx == 0.0 ? 0 : (ex == 0 ? -1022 : ex - 1022);
    const double inv = ldexp(1.0, -(g + SP_E1));
#pragma unroll
    for (int u = 0; u < NV; ++u) v[u] *= inv;
#pragma unroll
    for (int i = 0; i < SP_NS; ++i) {
        const double un = ldexp(1.0, 8 + 9 * i), ui = ldexp(1.0, -8 - 9 * i);
        double s[NV];
#pragma unroll
        for (int u = 0; u < NV; ++u) {
            s[u] = rint(v[u] * un) * ui;
            v[u] -= s[u];
        }
#pragma unroll
        for (int h = 0; h < NV / 2; ++h) {
            const __nv_bfloat162 p = __floats2bfloat162_rn((float)s[2 * h], (float)s[2 * h + 1]);
            *reinterpret_cast<__nv_bfloat162 *>(Xs + ((size_t)i * rowsX + R) * E_pad + j0 +
                                                h * SP_KC) = p;  // exact
        }
    }
    if (lane == 0) {
        float sc = 0.f;
        if (mx != 0.0)
            sc = g + SP_E1 > 127 ? __int_as_float(0x7f800000)
                                 : (g + SP_E1 < -149 ? 0.f : ldexpf(1.f, g + SP_E1));
        xsc[(size_t)c * rowsX + R] = sc;
    }
}

// Row exponents of A: rexp[(d n_rc + c) E + l] = e with 2^e just above the
// largest |A^d[l][j]| of the column chunk c (clamped to [-126, 127]).  A CTA
// takes 32 consecutive rows of the stacked blocks (a warp per row) and writes
// the exponents chunk by chunk, 32 adjacent bytes each, so that the product's
// slicers and readers read a chunk's exponents of consecutive rows together.
constexpr int RE_ROWS = 32;
__global__ void __launch_bounds__(32 * RE_ROWS)
k_row_exp(const float *__restrict__ A, int E, int n_steps, int n_rc, int8_t *__restrict__ rexp) {
    extern __shared__ int8_t ex[];  // [n_rc][RE_ROWS]
    const size_t g0 = (size_t)blockIdx.x * RE_ROWS, rows = (size_t)n_steps * E;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    {
        const int r = warp;
        const size_t g = g0 + r;
        const float *row = A + min(g, rows - 1) * E;
        for (int c = 0; c < n_rc && g < rows; ++c) {
            float m = 0.f;
#pragma unroll
            for (int u = 0; u < SP_RC / 32; ++u) {
                const int j = c * SP_RC + u * 32 + lane;
                if (j < E) m = fmaxf(m, fabsf(__ldg(row + j)));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) ex[c * RE_ROWS + r] = (int8_t)min(scale_exp(m), 127);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n_rc * RE_ROWS; t += blockDim.x) {
        const int r = t % RE_ROWS, c = t / RE_ROWS;
        const size_t g = g0 + r;
        if (g < rows) rexp[((g / E) * n_rc + c) * E + g % E] = ex[t];
    }
}

// ------------------------------------------------------------ main kernel
struct SplitArgs {
    const float *A;
    const float *xsc;
    const int8_t *rexp;
    double *part;
    int32_t *status;
    int E, n_steps, nrhs, rpad, lg_rpad, S, rowsX, n_sub, n_rc, dr_len;
};

// 32 consecutive entries j0 .. j0+31 of row `row` of block d (zero outside)
template <bool VEC>
__device__ __forceinline__ void load32(const float *A, int E, int d, int row, int j0,
                                       float4 (&v)[8]) {
    if (row >= E) {
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const float *p = A + ((size_t)d * E + row) * E + j0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int j = j0 + 4 * q;
        if (VEC)
            v[q] = j < E ? __ldg(reinterpret_cast<const float4 *>(p) + q)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
        else
            v[q] = make_float4(j < E ? __ldg(p + 4 * q) : 0.f, j + 1 < E ? __ldg(p + 4 * q + 1) : 0.f,
                               j + 2 < E ? __ldg(p + 4 * q + 2) : 0.f,
                               j + 3 < E ? __ldg(p + 4 * q + 3) : 0.f);
    }
}

// Pieces of 64 columns j are visited in the order (d, c), c = 0 .. n_sub-1
// for each block d; pieces 2p and 2p+1 of a block form scale chunk p.
struct PieceIter {
    int d, c;
    __device__ __forceinline__ void next(int n_sub) {
        if (++c == n_sub) {
            c = 0;
            ++d;
        }
    }
};

template <bool VEC>
__global__ void __launch_bounds__(SP_THREADS, 1)
k_toeplitz_split(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapA,
                 const SplitArgs a) {
    using Sh = SplitShape<VEC>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + Sh::OFF_BAR;
    const uint32_t bfull = bar0, bempty = bar0 + 16, afull = bar0 + 32, aempty = afull + 8 * Sh::NA,
                   accfull = aempty + 8 * Sh::NA, accempty = accfull + 16, drain = accempty + 16,
                   ffull = drain + 8, fempty = ffull + 8 * Sh::NF;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + Sh::OFF_MISC);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + Sh::OFF_MISC + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * SP_M;
    const int n0 = blockIdx.y * a.S;  // first step of the box
    const int d0 = blockIdx.z * a.dr_len;
    const int d1 = min(min(d0 + a.dr_len, a.n_steps), n0 + a.S);  // later blocks meet zero rows
    if (d0 >= d1) return;  // the reduction never reads this slice for these columns
    const int T = (d1 - d0) * a.n_sub;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(bfull + 8 * s, 1);
            mbar_init(bempty + 8 * s, 1);
            mbar_init(accfull + 8 * s, 1);
            mbar_init(accempty + 8 * s, SP_READERS / 32);
        }
        for (int s = 0; s < Sh::NA; ++s) {
            mbar_init(afull + 8 * s, SP_SLICERS / 32);
            mbar_init(aempty + 8 * s, 1);
        }
        for (int s = 0; s < Sh::NF; ++s) {
            mbar_init(ffull + 8 * s, 1);
            mbar_init(fempty + 8 * s, SP_SLICERS / 32);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_slot), SP_TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer: the five x-slice tiles of each piece (and its A tile)
            int issued = 0;
            PieceIter it{d0, 0};
            for (int t = 0; t < T; ++t, it.next(a.n_sub)) {
                if constexpr (Sh::NF > 0) {
                    const int f = t % Sh::NF;
                    if (!mbar_wait_bounded(fempty + 8 * f, ((t / Sh::NF) & 1) ^ 1, a.status, abort_flag,
                                           TC_WAIT_NS))
                        break;
                    const uint32_t fdst = sbase + Sh::OFF_F + f * Sh::F_BYTES;
                    mbar_expect_tx(ffull + 8 * f, Sh::F_BYTES);
                    // rows past E of the last row tile read the next block's rows (or
                    // the tensor's zero fill); the slicers zero them
                    tma_load_2d(fdst, &mapA, it.c * SP_KC, it.d * a.E + m0, ffull + 8 * f);
                    tma_load_2d(fdst + Sh::F_HALF, &mapA, it.c * SP_KC + 32, it.d * a.E + m0,
                                ffull + 8 * f);
                }
                const int s = t & 1;
                if (!mbar_wait_bounded(bempty + 8 * s, ((t >> 1) & 1) ^ 1, a.status, abort_flag,
                                       TC_WAIT_NS))
                    break;
                const uint32_t dst = sbase + Sh::OFF_B + s * SP_BSTAGE;
                const int y0 = (a.S + n0 - it.d) * a.rpad;
                mbar_expect_tx(bfull + 8 * s, SP_BSTAGE);
#pragma unroll
                for (int i = 0; i < SP_NS; ++i)
                    tma_load_2d(dst + i * SP_B_BYTES, &mapX, it.c * SP_KC, i * a.rowsX + y0,
                                bfull + 8 * s);
                issued = t + 1;
            }
            // the copies of the last two pieces have landed before the CTA may exit
            for (int t = max(0, issued - 2); t < issued; ++t)
                mbar_wait_bounded(bfull + 8 * (t & 1), (t >> 1) & 1, a.status, nullptr, TC_WAIT_NS);
            if constexpr (Sh::NF > 0)
                for (int t = max(0, issued - Sh::NF); t < issued; ++t)
                    mbar_wait_bounded(ffull + 8 * (t % Sh::NF), (t / Sh::NF) & 1, a.status, nullptr,
                                      TC_WAIT_NS);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer; accumulator buffer r & 1 for scale chunk r
            PieceIter it{d0, 0};
            int r = 0;
            for (int t = 0; t < T; ++t, it.next(a.n_sub)) {
                const bool first = it.c % SP_PPC == 0,
                           last = it.c % SP_PPC == SP_PPC - 1 || it.c + 1 == a.n_sub;
                const int buf = r & 1;
                if (first && !mbar_wait_bounded(accempty + 8 * buf, ((r >> 1) & 1) ^ 1, a.status,
                                                abort_flag, TC_WAIT_NS))
                    break;
                if (!mbar_wait_bounded(bfull + 8 * (t & 1), (t >> 1) & 1, a.status, abort_flag,
                                       TC_WAIT_NS))
                    break;
                tc_fence_after();
                const uint32_t bst = sbase + Sh::OFF_B + (t & 1) * SP_BSTAGE;
                bool ok = true;
                for (int i = 0; i < SP_NS && ok; ++i) {
                    const int u = SP_NS * t + i, slot = u % Sh::NA;
                    if (!mbar_wait_bounded(afull + 8 * slot, (u / Sh::NA) & 1, a.status, abort_flag,
                                           TC_WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ad = smem_desc_sw128(sbase + slot * SP_A_BYTES);
                    // A slice i against x slices 0 .. 3-i: the levels i .. 3 are
                    // adjacent accumulators and the x slices adjacent tiles, so the
                    // products are one MMA of N = 64 (4 - i) (the i = 0 MMA of a
                    // chunk's first k step overwrites all four levels)
                    const int nlev = SP_NL - i;
                    if (nlev > 0) {
                        const uint32_t dt = tmem + (uint32_t)(buf * SP_NL * SP_N + i * SP_N);
                        const uint64_t bd = smem_desc_sw128(bst);
                        const uint32_t idn = idesc_bf16(SP_M, SP_N * nlev);
#pragma unroll
                        for (int kk = 0; kk < SP_KC / 16; ++kk)  // 16 bf16 = 32 bytes: +2
                            umma_bf16(dt, ad + 2 * kk, bd + 2 * kk, idn,
                                      (first && i == 0 && kk == 0) ? 0u : 1u);
                    }
                    {  // level 4: x slice 4-i into the level-3 accumulator
                        const int j = SP_NS - 1 - i;
                        const uint32_t dt =
                            tmem + (uint32_t)(buf * SP_NL * SP_N + (SP_NL - 1) * SP_N);
                        const uint64_t bd = smem_desc_sw128(bst + j * SP_B_BYTES);
#pragma unroll
                        for (int kk = 0; kk < SP_KC / 16; ++kk)
                            umma_bf16(dt, ad + 2 * kk, bd + 2 * kk, SP_IDESC, 1u);
                    }
                    umma_commit(aempty + 8 * slot);  // the slot is free once read
                }
                if (!ok) break;
                umma_commit(bempty + 8 * (t & 1));
                if (last) {
                    umma_commit(accfull + 8 * buf);
                    ++r;
                }
            }
            umma_commit(drain);  // completes when every MMA issued above has
        }
        __syncwarp();
    } else {
        if (warp < 2 + SP_SLICERS / 32) {
            // ------------------------------------------------------ slicers
            // slicer (q, h) owns tile row 32q + lane and the 32 columns j of half h
            const int sw = warp - 2, q = sw & 3, h = sw >> 2;
            const int rl = 32 * q + lane, row = m0 + rl, jh = 32 * h;
            // the current piece in registers; the next two pieces are prefetched
            // into L2 (no registers) and the next one is loaded as soon as the
            // current one is sliced
            // (with TA: the piece's row segment from the staged A tile instead)
            float4 cur[8];
            if constexpr (Sh::NF == 0) load32<VEC>(a.A, a.E, d0, row, jh, cur);
            PieceIter it{d0, 0};
            float2 inv = make_float2(0.f, 0.f);
            int e_next = row < a.E ? (int)a.rexp[(size_t)d0 * a.n_rc * a.E + row] : 0;
            for (int t = 0; t < T; ++t) {
                PieceIter nx = it;
                nx.next(a.n_sub);
                if constexpr (Sh::NF > 0) {  // this row's 128 bytes of half h, chunk k at k ^ (rl % 8)
                    const int f = t % Sh::NF;
                    const bool ok = mbar_wait_bounded(ffull + 8 * f, (t / Sh::NF) & 1, a.status,
                                                      abort_flag, TC_WAIT_NS);
                    const unsigned char *seg =
                        smem + Sh::OFF_F + f * Sh::F_BYTES + h * Sh::F_HALF + rl * 128;
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        cur[k] = ok && row < a.E
                                     ? *reinterpret_cast<const float4 *>(seg + ((k ^ (rl & 7)) << 4))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                if (Sh::NF == 0 && row < a.E) {  // this thread's 128-byte line of pieces t+1 and t+2
                    PieceIter n2 = nx;
#pragma unroll
                    for (int ahead = 1; ahead <= 2; ++ahead) {
                        const int j2 = n2.c * SP_KC + jh;
                        if (t + ahead < T && j2 < a.E)
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(
                                a.A + ((size_t)n2.d * a.E + row) * a.E + j2));
                        n2.next(a.n_sub);
                    }
                }
                if (it.c % SP_PPC == 0) {  // a new scale chunk: this row's exponent
                    const float iv = pow2f(-(e_next + SP_E1));
                    inv = make_float2(iv, iv);
                }
                if (t + 1 < T && nx.c % SP_PPC == 0)  // the next chunk's, loaded a piece ahead
                    e_next = row < a.E
                                 ? (int)a.rexp[((size_t)nx.d * a.n_rc + nx.c / SP_PPC) * a.E + row]
                                 : 0;
                float2 v[16];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    v[2 * i] = __fmul2_rn(make_float2(cur[i].x, cur[i].y), inv);
                    v[2 * i + 1] = __fmul2_rn(make_float2(cur[i].z, cur[i].w), inv);
                }
                if constexpr (Sh::NF > 0) {
                    // the staged tile is released only once its values are in
                    // registers (v depends on every load), so that the next TMA
                    // cannot overwrite a load still in flight
                    __syncwarp();
                    if (lane == 0) mbar_arrive(fempty + 8 * (t % Sh::NF));
                }
#pragma unroll
                for (int i = 0; i < SP_NS; ++i) {
                    const int u = SP_NS * t + i, slot = u % Sh::NA;
                    const bool ok = mbar_wait_bounded(aempty + 8 * slot, ((u / Sh::NA) & 1) ^ 1,
                                                      a.status, abort_flag, TC_WAIT_NS);
                    // slice i: round to a multiple of 2^(-8-9i) (|D| <= 256, exact in bf16)
                    const float ci = 1.5f * __int_as_float((127 + 15 - 9 * i) << 23);
                    const float2 C = make_float2(ci, ci);
                    unsigned char *tile = smem + slot * SP_A_BYTES;
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {  // 8 columns (16 bytes) at a time
                        uint32_t w[4];
#pragma unroll
                        for (int p2 = 0; p2 < 4; ++p2) {
                            float2 &vp = v[4 * qq + p2];
                            const float2 s = sub2(__fadd2_rn(vp, C), C);
                            if (i + 1 < SP_NS) vp = sub2(vp, s);
                            const __nv_bfloat162 b = __floats2bfloat162_rn(s.x, s.y);
                            w[p2] = *reinterpret_cast<const uint32_t *>(&b);
                        }
                        if (ok)
                            *reinterpret_cast<uint4 *>(tile + sw128_offset_b16(rl, jh + 8 * qq)) =
                                make_uint4(w[0], w[1], w[2], w[3]);
                    }
                    if (ok) fence_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(afull + 8 * slot);
                }
                if (Sh::NF == 0 && t + 1 < T) load32<VEC>(a.A, a.E, nx.d, row, nx.c * SP_KC + jh, cur);
                it = nx;
            }
        } else {
            // --------------------------------------------------- read-back
            // reader (q, ch) owns TMEM lane 32q + lane = tile row and the 32 output
            // columns of half ch; it reads every 128-column chunk's accumulators
            const int ew = warp - 2 - SP_SLICERS / 32, q = warp & 3, ch = ew >> 2;
            const int rl = 32 * q + lane, row = m0 + rl, jc = 32 * ch;
            // running double-float sums of its 32 columns: high parts in registers,
            // low parts in shared memory (consecutive rows: conflict-free)
            float2 ah[16];
            float2 *al = reinterpret_cast<float2 *>(smem + Sh::OFF_AL) + (jc >> 1) * SP_M + rl;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                ah[i] = make_float2(0.f, 0.f);
                al[i * SP_M] = make_float2(0.f, 0.f);
            }
            const float2 C16 = make_float2(192.f, 192.f);  // rounds to multiples of 2^-16
            const int n_read = (d1 - d0) * a.n_rc;
            int d = d0, pch = 0;
            for (int r = 0; r < n_read; ++r) {
                const int buf = r & 1;
                const int e = row < a.E ? (int)a.rexp[((size_t)d * a.n_rc + pch) * a.E + row] : 0;
                const float rs = pow2f(e + SP_E1);
                const bool ok = mbar_wait_bounded(accfull + 8 * buf, (r >> 1) & 1, a.status,
                                                  abort_flag, TC_WAIT_NS);
                tc_fence_after();
                if (ok) {
                    // x scales of the 32 columns (the table has S zero steps in front
                    // and 64 zero rows behind, so every window stays inside it)
                    const float *cs = a.xsc + (size_t)pch * a.rowsX + (a.S + n0 - d) * a.rpad + jc;
                    const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) +
                                        (uint32_t)(buf * SP_NL * SP_N + jc);
                    const float2 rs2 = make_float2(rs, rs);
#pragma unroll
                    for (int g = 0; g < 4; ++g) {  // 8 columns per round trip to tensor memory
                        uint32_t L[SP_NL][8];
#pragma unroll
                        for (int l = 0; l < SP_NL; ++l) tmem_ld8_nowait(tb + l * SP_N + 8 * g, L[l]);
                        float cgs[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) cgs[u] = __ldg(cs + 8 * g + u);
                        tmem_wait_ld();
#pragma unroll
                        for (int pp = 0; pp < 4; ++pp) {
                            const int ia = 4 * g + pp;  // column pair
                            const float2 cg = make_float2(cgs[2 * pp], cgs[2 * pp + 1]);
                            const float2 l0 = make_float2(__uint_as_float(L[0][2 * pp]), __uint_as_float(L[0][2 * pp + 1]));
                            const float2 l1 = make_float2(__uint_as_float(L[1][2 * pp]), __uint_as_float(L[1][2 * pp + 1]));
                            const float2 l2 = make_float2(__uint_as_float(L[2][2 * pp]), __uint_as_float(L[2][2 * pp + 1]));
                            const float2 l3 = make_float2(__uint_as_float(L[3][2 * pp]), __uint_as_float(L[3][2 * pp + 1]));
                            const float2 l1h = sub2(__fadd2_rn(l1, C16), C16);
                            const float2 hi = __fadd2_rn(l0, l1h);
                            const float2 lo = __fadd2_rn(sub2(l1, l1h), l2);
                            float2 hh = __fadd2_rn(hi, lo);
                            float2 bb = sub2(hh, hi);
                            float2 ll =
                                __fadd2_rn(__fadd2_rn(sub2(hi, sub2(hh, bb)), sub2(lo, bb)), l3);
                            const float2 sc = __fmul2_rn(rs2, cg);
                            hh = __fmul2_rn(hh, sc);
                            ll = __fmul2_rn(ll, sc);
                            // (ah, al) += (hh, ll): error-free sum of the high parts, then
                            // renormalised so that |al| stays below half an ulp of ah
                            const float2 s = __fadd2_rn(ah[ia], hh);
                            bb = sub2(s, ah[ia]);
                            float2 err = __fadd2_rn(sub2(ah[ia], sub2(s, bb)), sub2(hh, bb));
                            err = __fadd2_rn(err, __fadd2_rn(al[ia * SP_M], ll));
                            const float2 nh = __fadd2_rn(s, err);
                            ah[ia] = nh;
                            al[ia * SP_M] = sub2(err, sub2(nh, s));
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(accempty + 8 * buf);
                if (++pch == a.n_rc) {
                    pch = 0;
                    ++d;
                }
            }
            if (!*abort_flag && row < a.E) {  // partial sums of this slice of blocks
                const int zslice = blockIdx.z;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
#pragma unroll
                    for (int e2 = 0; e2 < 2; ++e2) {
                        const int col = jc + 2 * i + e2;
                        const int k = n0 + (col >> a.lg_rpad), rr = col & (a.rpad - 1);
                        if (k < a.n_steps && rr < a.nrhs) {
                            const float2 lw = al[i * SP_M];
                            const double val = e2 == 0 ? (double)ah[i].x + (double)lw.x
                                                       : (double)ah[i].y + (double)lw.y;
                            a.part[(((size_t)zslice * a.nrhs + rr) * a.n_steps + k) * a.E + row] =
                                val;
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        // every MMA has completed before the tensor memory is released
        mbar_wait_bounded(drain, 0, a.status, nullptr, TC_WAIT_NS);
        tc_fence_after();
        tmem_dealloc(tmem, SP_TMEM_COLS);
    }
}

// y = beta y + sum of the slices holding blocks d <= k, or y = f - that sum
__global__ void k_split_reduce(const double *__restrict__ part, int E, int n_steps, int nrhs,
                               int dr_len, int mode, const double *f, double beta, double *y) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)nrhs * n_steps * E;
    if (idx >= total) return;
    const int k = (int)((idx / E) % n_steps);
    double s = 0.0;
    for (int z = 0; z * dr_len <= k; ++z) s += part[(size_t)z * total + idx];
    if (mode == DF_RESIDUAL)
        y[idx] = f[idx] - s;
    else
        y[idx] = beta == 0.0 ? s : fma(beta, y[idx], s);
}

// ------------------------------------------------------------------ host ---
struct SplitPlan {
    int rpad, lg_rpad, S, n_box, rowsX, n_sub, n_rc, E_pad, row_tiles, dr_len, n_z, nrhs_g;
    size_t xs_bytes, xsc_bytes, rexp_bytes, part_bytes;
};

static SplitPlan split_plan(int64_t E, int n_steps, int nrhs) {
    SplitPlan p{};
    p.nrhs_g = std::min(nrhs, 64);
    p.rpad = 1;
    while (p.rpad < p.nrhs_g) p.rpad *= 2;
    while ((1 << p.lg_rpad) < p.rpad) ++p.lg_rpad;
    p.S = SP_N / p.rpad;
    p.n_box = (n_steps + p.S - 1) / p.S;
    p.rowsX = (p.S + n_steps) * p.rpad + SP_N;  // + 64 zero rows: windows stay inside
    p.n_sub = (int)((E + SP_KC - 1) / SP_KC);
    p.n_rc = (int)((E + SP_RC - 1) / SP_RC);
    p.E_pad = p.n_rc * SP_RC;
    p.row_tiles = (int)((E + SP_M - 1) / SP_M);
    int64_t wb = 0;  // (row tile, box, block) triples
    for (int b = 0; b < p.n_box; ++b) wb += std::min(n_steps, b * p.S + p.S);
    wb *= p.row_tiles;
    const int64_t target = 4 * 152;  // about four waves of one CTA per SM
    p.dr_len = (int)std::max<int64_t>(1, std::min<int64_t>(64, (wb + target - 1) / target));
    p.dr_len = std::min(p.dr_len, n_steps);
    p.n_z = (n_steps + p.dr_len - 1) / p.dr_len;
    p.xs_bytes = align256((size_t)SP_NS * p.rowsX * p.E_pad * 2);
    p.xsc_bytes = align256((size_t)p.n_rc * p.rowsX * 4);
    p.rexp_bytes = align256((size_t)n_steps * E * p.n_rc);
    p.part_bytes = align256((size_t)p.n_z * p.nrhs_g * n_steps * E * sizeof(double));
    return p;
}

size_t toeplitz_split_bytes(int64_t E, int32_t n_steps, int32_t nrhs) {
    const SplitPlan p = split_plan(E, n_steps, nrhs);
    return p.xs_bytes + p.xsc_bytes + p.rexp_bytes + p.part_bytes;
}

template <class XT>
static stb_status split_run(const float *A, int64_t E, int32_t n_steps, int32_t nrhs, const XT *x,
                            int mode, const double *f, double beta, double *y, void *scratch,
                            int32_t *status, bool a_exp_ready, cudaStream_t s) {
    if (E < 1 || E > 65535 || n_steps < 1 || nrhs < 1)
        return fail(STB_ERR_INVALID_ARG, "split product: need 1 <= E <= 65535, n_steps, nrhs >= 1");
    const SplitPlan p = split_plan(E, n_steps, nrhs);
    char *sc = static_cast<char *>(scratch);
    __nv_bfloat16 *Xs = reinterpret_cast<__nv_bfloat16 *>(sc);
    float *xsc = reinterpret_cast<float *>(sc + p.xs_bytes);
    int8_t *rexp = reinterpret_cast<int8_t *>(sc + p.xs_bytes + p.xsc_bytes);
    double *part = reinterpret_cast<double *>(sc + p.xs_bytes + p.xsc_bytes + p.rexp_bytes);
    CUtensorMap mapX, mapA;
    stb_status st = tc_make_map_2d(&mapX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Xs,
                                   (uint64_t)SP_NS * p.rowsX, (uint64_t)p.E_pad, SP_KC, SP_N);
    if (st) return st;
    const bool vec = E % 4 == 0 && reinterpret_cast<uintptr_t>(A) % 16 == 0;
    if (vec) {  // A as n_steps E rows of E FP32 columns; boxes of 128 rows x 32 columns
        if ((st = tc_make_map_2d(&mapA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, A,
                                 (uint64_t)n_steps * E, (uint64_t)E, 32, SP_M)))
            return st;
    } else {
        mapA = mapX;  // not read
    }
    const auto kern = vec ? k_toeplitz_split<true> : k_toeplitz_split<false>;
    const size_t smem = vec ? SplitShape<true>::SMEM : SplitShape<false>::SMEM;
    STB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (!a_exp_ready) {  // row exponents of every column chunk of A (one pass over the blocks)
        const size_t rows = (size_t)n_steps * E;
        count_launch(s);
        k_row_exp<<<(unsigned)((rows + RE_ROWS - 1) / RE_ROWS), 32 * RE_ROWS, (size_t)p.n_rc * RE_ROWS, s>>>(
            A, (int)E, n_steps, p.n_rc, rexp);
        if ((st = check_launch("k_row_exp"))) return st;
    }
    const size_t stride = (size_t)n_steps * E;  // one right-hand side
    for (int r0 = 0; r0 < nrhs; r0 += 64) {
        const int ng = std::min(64, nrhs - r0);
        const size_t warps = (size_t)p.rowsX * p.n_rc;
        count_launch(s);
        k_split_x<XT><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(
            x + r0 * stride, (int)E, p.E_pad, n_steps, ng, p.rpad, p.S, p.rowsX, p.n_rc, Xs, xsc);
        if ((st = check_launch("k_split_x"))) return st;
        SplitArgs args{A, xsc, rexp, part, status, (int)E, n_steps, ng, p.rpad, p.lg_rpad, p.S,
                       p.rowsX, p.n_sub, p.n_rc, p.dr_len};
        const dim3 grid((unsigned)p.row_tiles, (unsigned)p.n_box, (unsigned)p.n_z);
        count_launch(s);
        kern<<<grid, SP_THREADS, smem, s>>>(mapX, mapA, args);
        if ((st = check_launch("k_toeplitz_split"))) return st;
        const size_t total = (size_t)ng * stride;
        count_launch(s);
        k_split_reduce<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
            part, (int)E, n_steps, ng, p.dr_len, mode, f ? f + r0 * stride : nullptr, beta,
            y + r0 * stride);
        if ((st = check_launch("k_split_reduce"))) return st;
    }
    return STB_OK;
}

stb_status toeplitz_split(const float *A, int64_t E, int32_t n_steps, int32_t nrhs, const double *x,
                          int mode, const double *f, double beta, double *y, void *scratch,
                          int32_t *status, cudaStream_t s) {
    return split_run<double>(A, E, n_steps, nrhs, x, mode, f, beta, y, scratch, status, false, s);
}

stb_status toeplitz_split_f32x(const float *A, int64_t E, int32_t n_steps, int32_t nrhs,
                               const float *x, int mode, const double *f, double beta, double *y,
                               void *scratch, int32_t *status, bool a_exp_ready, cudaStream_t s) {
    return split_run<float>(A, E, n_steps, nrhs, x, mode, f, beta, y, scratch, status, a_exp_ready,
                            s);
}


// ===================================================================== panel
// Far history of a panel of PB = 8 time steps of the march (FP32 accuracy):
//   part[z][r][c][l] = sum_{d in slice z} V^d[l,:] x_r^{kp+c-d},  0 <= kp+c-d < kp,
// on the tensor cores.  Both operands are split into three bf16 slices of
// floating (per element) exponent, a = a0 + a1 + a2 exactly for an FP32 a
// (8 + 8 + 8 significant bits, round to nearest), and the six products with
// i + j <= 2 are accumulated in FP32 tensor memory, one accumulator per level
// s = i + j (adjacent, so that A slice i meets x slices 0 .. 2-i in one MMA
// of N (3 - i) columns): about 2^-22 relative per term.  The tensor cores
// round their FP32 sums toward zero, a bias of about 2^-24 of the
// accumulator per MMA that grows with the length of the sum, so the
// accumulators are restarted every PN_G pieces (at most 48 MMAs into a level)
// and the group sums are added in registers (round to nearest), two sets
// alternating so that the MMAs of one group overlap the read-back of the one
// before.  The
// x slices are kept step-major, Xf[i][(PB + m) rpad + r][j], and filled
// panel by panel (steps not yet solved stay zero), so the B tile of block d
// is the contiguous window of N = 8 rpad rows (at least 16) starting at
// (PB + kp - d) rpad.
// The FP32 A tiles (128 rows x 64 columns of a block) come by TMA, in two
// 32-column halves with the 128-byte swizzle, into a ring of FP32 stages;
// the workers slice them from shared memory into the bf16 slot ring.
constexpr int PN_NS = 3;
constexpr int PN_NA = 3;           // A-slice slots (one piece: its slicing is quick from shared memory)
constexpr int PN_PB = 8;           // steps per panel
constexpr int PN_MAX_Z = 64;       // slices of the block range
constexpr int PN_G = 4;            // pieces per tensor-memory accumulation group
constexpr int PN_THREADS = SP_THREADS;  // warp 0 TMA, warp 1 MMA, 16 workers

template <int N>
struct PanelShape {
    static constexpr int NB = N == 64 ? 2 : 4;    // x-slice stages
    static constexpr int NF = 3;                  // FP32 A stages
    static constexpr uint32_t B_BYTES = N * 128;                  // one slice tile
    static constexpr uint32_t BSTAGE = PN_NS * B_BYTES;
    static constexpr uint32_t F_HALF = SP_M * 128;                // 32 FP32 columns
    static constexpr uint32_t F_BYTES = 2 * F_HALF;               // one FP32 A tile
    static constexpr uint32_t OFF_F = PN_NA * SP_A_BYTES;
    static constexpr uint32_t OFF_B = OFF_F + NF * F_BYTES;
    static constexpr uint32_t OFF_BAR = OFF_B + NB * BSTAGE;
    static constexpr int NBAR = 2 * NB + 2 * PN_NA + 1 + 4 + 2 * NF;
    static constexpr uint32_t OFF_MISC = OFF_BAR + NBAR * 8;
    static constexpr size_t SMEM = OFF_MISC + 16 + 1024;
    // two sets of three level accumulators (a power of two of at least 32 columns)
    static constexpr uint32_t TMEM_COLS = 6 * N <= 32 ? 32 : 6 * N <= 64 ? 64 : 6 * N <= 128 ? 128
                                        : 6 * N <= 256 ? 256 : 512;
    static constexpr int NQ = N / 4;  // columns read back by each worker
    static_assert(SMEM <= 232448, "shared memory of the panel product");
};

struct PanelArgs {
    const float *V;
    float *part;
    int32_t *status;
    int E, nrhs, rpad, rowsX, n_chunks, kp, nb, d_lo, d_end, dr_len;
};

// three floating bf16 slices of a float pair (exact)
__device__ __forceinline__ void split3_bf16(float2 v, uint32_t &w0, uint32_t &w1, uint32_t &w2) {
    __nv_bfloat162 b = __floats2bfloat162_rn(v.x, v.y);
    w0 = *reinterpret_cast<const uint32_t *>(&b);
    float2 r = sub2(v, __bfloat1622float2(b));
    b = __floats2bfloat162_rn(r.x, r.y);
    w1 = *reinterpret_cast<const uint32_t *>(&b);
    r = sub2(r, __bfloat1622float2(b));
    b = __floats2bfloat162_rn(r.x, r.y);
    w2 = *reinterpret_cast<const uint32_t *>(&b);
}

// Xf rows of steps [m_lo, m_hi), right-hand sides r < nrhs, j < E (the rest
// of Xf is zero and stays zero)
__global__ void k_panel_split_x(const float *__restrict__ x, int E, int E_pad, int n_steps,
                                int nrhs, int rpad, int rowsX, int m_lo, int m_hi,
                                __nv_bfloat16 *__restrict__ Xf) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // pair of columns
    const int half = (E + 1) / 2;
    const size_t total = (size_t)(m_hi - m_lo) * nrhs * half;
    if (i >= total) return;
    const int jp = (int)(i % half), r = (int)((i / half) % nrhs), m = m_lo + (int)(i / ((size_t)half * nrhs));
    const int j = 2 * jp;
    const float *xr = x + ((size_t)r * n_steps + m) * E;
    const float2 v = make_float2(xr[j], j + 1 < E ? xr[j + 1] : 0.f);
    uint32_t w[3];
    split3_bf16(v, w[0], w[1], w[2]);
    const size_t R = (size_t)(PN_PB + m) * rpad + r;
#pragma unroll
    for (int s = 0; s < PN_NS; ++s)
        *reinterpret_cast<uint32_t *>(Xf + ((size_t)s * rowsX + R) * E_pad + j) = w[s];
}

template <int N>
__global__ void __launch_bounds__(PN_THREADS, 1)
k_toeplitz_panel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapA,
                 const PanelArgs a) {
    using Sh = PanelShape<N>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bfull = sbase + Sh::OFF_BAR, bempty = bfull + 8 * Sh::NB,
                   afull = bempty + 8 * Sh::NB, aempty = afull + 8 * PN_NA, done = aempty + 8 * PN_NA,
                   accf = done + 8, acce = accf + 16, ffull = acce + 16, fempty = ffull + 8 * Sh::NF;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + Sh::OFF_MISC);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + Sh::OFF_MISC + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const int m0 = blockIdx.x * SP_M;
    const int d0 = a.d_lo + blockIdx.z * a.dr_len;
    const int d1 = min(d0 + a.dr_len, a.d_end);
    if (d0 >= d1) return;
    const int T = (d1 - d0) * a.n_chunks;

    if (threadIdx.x == 0) {
        for (int s = 0; s < Sh::NB; ++s) {
            mbar_init(bfull + 8 * s, 1);
            mbar_init(bempty + 8 * s, 1);
        }
        for (int s = 0; s < Sh::NF; ++s) {
            mbar_init(ffull + 8 * s, 1);
            mbar_init(fempty + 8 * s, SP_WORKERS / 32);
        }
        for (int s = 0; s < PN_NA; ++s) {
            mbar_init(afull + 8 * s, SP_WORKERS / 32);
            mbar_init(aempty + 8 * s, 1);
        }
        mbar_init(done, 1);  // (panel)
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf + 8 * b, 1);
            mbar_init(acce + 8 * b, SP_WORKERS / 32);
        }
        *abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_slot), Sh::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer of the FP32 A tiles and the x slices
            int issued = 0;
            PieceIter it{d0, 0};
            for (int t = 0; t < T; ++t, it.next(a.n_chunks)) {
                const int d = it.d, c = it.c;
                const int f = t % Sh::NF;
                if (!mbar_wait_bounded(fempty + 8 * f, ((t / Sh::NF) & 1) ^ 1, a.status, abort_flag,
                                       TC_WAIT_NS))
                    break;
                const uint32_t fdst = sbase + Sh::OFF_F + f * Sh::F_BYTES;
                mbar_expect_tx(ffull + 8 * f, Sh::F_BYTES);
                // rows past E of the last row tile read the next block's rows
                // (or the tensor's zero fill), never stored
                tma_load_2d(fdst, &mapA, c * SP_KC, d * a.E + m0, ffull + 8 * f);
                tma_load_2d(fdst + Sh::F_HALF, &mapA, c * SP_KC + 32, d * a.E + m0, ffull + 8 * f);
                const int s = t % Sh::NB, u = t / Sh::NB;
                if (!mbar_wait_bounded(bempty + 8 * s, (u & 1) ^ 1, a.status, abort_flag, TC_WAIT_NS))
                    break;
                const uint32_t dst = sbase + Sh::OFF_B + s * Sh::BSTAGE;
                const int y0 = (PN_PB + a.kp - d) * a.rpad;
                mbar_expect_tx(bfull + 8 * s, Sh::BSTAGE);
#pragma unroll
                for (int i = 0; i < PN_NS; ++i)
                    tma_load_2d(dst + i * Sh::B_BYTES, &mapX, c * SP_KC, i * a.rowsX + y0, bfull + 8 * s);
                issued = t + 1;
            }
            // the copies still in flight have landed before the CTA may exit
            for (int t = max(0, issued - Sh::NB); t < issued; ++t)
                mbar_wait_bounded(bfull + 8 * (t % Sh::NB), (t / Sh::NB) & 1, a.status, nullptr,
                                  TC_WAIT_NS);
            for (int t = max(0, issued - Sh::NF); t < issued; ++t)
                mbar_wait_bounded(ffull + 8 * (t % Sh::NF), (t / Sh::NF) & 1, a.status, nullptr,
                                  TC_WAIT_NS);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer: group g of PN_G pieces into accumulator g % 2
            for (int t = 0; t < T; ++t) {
                const int s = t % Sh::NB, g = t / PN_G, b = g & 1;
                const bool first = t % PN_G == 0;
                if (first && g >= 2) {  // the workers have read group g - 2 back
                    if (!mbar_wait_bounded(acce + 8 * b, ((g >> 1) - 1) & 1, a.status, abort_flag,
                                           TC_WAIT_NS))
                        break;
                    tc_fence_after();
                }
                if (!mbar_wait_bounded(bfull + 8 * s, (t / Sh::NB) & 1, a.status, abort_flag, TC_WAIT_NS))
                    break;
                tc_fence_after();
                const uint32_t bst = sbase + Sh::OFF_B + s * Sh::BSTAGE;
                bool ok = true;
                for (int i = 0; i < PN_NS; ++i) {
                    const int u = PN_NS * t + i, slot = u % PN_NA;
                    if (!mbar_wait_bounded(afull + 8 * slot, (u / PN_NA) & 1, a.status, abort_flag,
                                           TC_WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ad = smem_desc_sw128(sbase + slot * SP_A_BYTES);
                    // levels i .. 2 of set b from x slices 0 .. 2-i (the i = 0 MMA
                    // of a group's first k step overwrites all three levels)
                    const uint32_t dt = tmem + (uint32_t)((3 * b + i) * N);
                    const uint64_t bd = smem_desc_sw128(bst);
                    const uint32_t idn = idesc_bf16(SP_M, N * (PN_NS - i));
#pragma unroll
                    for (int kk = 0; kk < SP_KC / 16; ++kk)
                        umma_bf16(dt, ad + 2 * kk, bd + 2 * kk, idn,
                                  (first && i == 0 && kk == 0) ? 0u : 1u);
                    umma_commit(aempty + 8 * slot);
                }
                if (!ok) break;
                umma_commit(bempty + 8 * s);
                if (t % PN_G == PN_G - 1 || t == T - 1) umma_commit(accf + 8 * b);
            }
            umma_commit(done);
        }
        __syncwarp();
    } else {
        // workers: slice the A chunks (three floating bf16 slices); worker
        // (q, c4) owns tile row 32q + lane and the 16 columns j of quarter c4
        const int q = warp & 3, c4 = (warp - 2) >> 2;
        const int rl = 32 * q + lane, row = m0 + rl, jq = 16 * c4;  // jq: first column
        // and reads back columns [c4 NQ, c4 NQ + NQ) of the group sums
        float sum[Sh::NQ];
#pragma unroll
        for (int i = 0; i < Sh::NQ; ++i) sum[i] = 0.f;
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(c4 * Sh::NQ);
        auto read_group = [&](int g) {
            const int b = g & 1;
            bool ok = mbar_wait_bounded(accf + 8 * b, (g >> 1) & 1, a.status, abort_flag, TC_WAIT_NS);
            ok = __all_sync(0xffffffffu, ok);
            tc_fence_after();
            if (ok) {  // the three levels, at most 8 columns at a time
                constexpr int W = Sh::NQ < 8 ? Sh::NQ : 8;
#pragma unroll
                for (int c0 = 0; c0 < Sh::NQ; c0 += W) {
                    uint32_t v[3][W];
#pragma unroll
                    for (int l = 0; l < 3; ++l) {
                        const uint32_t ta = tl + (uint32_t)((3 * b + l) * N + c0);
                        if constexpr (W == 8) tmem_ld8_nowait(ta, v[l]);
                        else tmem_ld4_nowait(ta, v[l]);
                    }
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < W; ++i)
                        sum[c0 + i] += (__uint_as_float(v[2][i]) + __uint_as_float(v[1][i])) +
                                       __uint_as_float(v[0][i]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce + 8 * b);
        };
        for (int t = 0; t < T; ++t) {
            if (t % PN_G == 0 && t >= 2 * PN_G) read_group(t / PN_G - 2);
            // this thread's 16 FP32 values of the staged A tile: half c4 / 2,
            // 16-byte chunks 4 (c4 % 2) .. +3 of row rl, stored at chunk ^ (rl % 8)
            float4 cur[4];
            {
                const int f = t % Sh::NF;
                const bool ok = mbar_wait_bounded(ffull + 8 * f, (t / Sh::NF) & 1, a.status,
                                                  abort_flag, TC_WAIT_NS);
                const unsigned char *half =
                    smem + Sh::OFF_F + f * Sh::F_BYTES + (c4 >> 1) * Sh::F_HALF + rl * 128;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    cur[k] = ok ? *reinterpret_cast<const float4 *>(
                                      half + (((4 * (c4 & 1) + k) ^ (rl & 7)) << 4))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            uint32_t w[PN_NS][8];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                split3_bf16(make_float2(cur[i].x, cur[i].y), w[0][2 * i], w[1][2 * i], w[2][2 * i]);
                split3_bf16(make_float2(cur[i].z, cur[i].w), w[0][2 * i + 1], w[1][2 * i + 1],
                            w[2][2 * i + 1]);
            }
            // the staged tile is released only once its values are consumed (the
            // slices depend on every load): the next TMA into it cannot race a load
            __syncwarp();
            if (lane == 0) mbar_arrive(fempty + 8 * (t % Sh::NF));
#pragma unroll
            for (int i = 0; i < PN_NS; ++i) {
                const int u = PN_NS * t + i, slot = u % PN_NA;
                const bool ok = mbar_wait_bounded(aempty + 8 * slot, ((u / PN_NA) & 1) ^ 1, a.status,
                                                  abort_flag, TC_WAIT_NS);
                if (ok) {
                    unsigned char *tile = smem + slot * SP_A_BYTES;
#pragma unroll
                    for (int qq = 0; qq < 2; ++qq)
                        *reinterpret_cast<uint4 *>(tile + sw128_offset_b16(rl, jq + 8 * qq)) =
                            make_uint4(w[i][4 * qq], w[i][4 * qq + 1], w[i][4 * qq + 2], w[i][4 * qq + 3]);
                    fence_async_smem();
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(afull + 8 * slot);
            }
        }
        // the last two groups, then the row's NQ columns of the slice's sum
        const int n_groups = (T + PN_G - 1) / PN_G;
        for (int g = max(0, n_groups - 2); g < n_groups; ++g) read_group(g);
        if (row < a.E && !*abort_flag) {
#pragma unroll
            for (int i = 0; i < Sh::NQ; ++i) {
                const int col = c4 * Sh::NQ + i, cc = col / a.rpad, r = col % a.rpad;
                if (cc < a.nb && r < a.nrhs)
                    a.part[(((size_t)blockIdx.z * a.nrhs + r) * PN_PB + cc) * a.E + row] = sum[i];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        mbar_wait_bounded(done, 0, a.status, nullptr, TC_WAIT_NS);
        tc_fence_after();
        tmem_dealloc(tmem, Sh::TMEM_COLS);
    }
}

struct PanelPlan {
    int rpad, N, rowsX, n_chunks, E_pad, row_tiles;
    size_t xf_bytes;
};
static PanelPlan panel_plan(int64_t E, int n_steps, int nrhs) {
    PanelPlan p{};
    p.rpad = 1;
    while (p.rpad < nrhs) p.rpad *= 2;
    p.N = std::max(16, PN_PB * p.rpad);
    p.rowsX = (PN_PB + n_steps) * p.rpad + p.N;  // + N zero rows: windows never leave a slice
    p.n_chunks = (int)((E + SP_KC - 1) / SP_KC);
    p.E_pad = p.n_chunks * SP_KC;
    p.row_tiles = (int)((E + SP_M - 1) / SP_M);
    p.xf_bytes = align256((size_t)PN_NS * p.rowsX * p.E_pad * 2);
    return p;
}

bool panel_tc_supported(int32_t nrhs) { return nrhs >= 1 && nrhs <= 8; }
bool panel_tc_blocks_ok(const float *V, int64_t E) {  // TMA rows of V: 16-byte aligned
    return E % 4 == 0 && reinterpret_cast<uintptr_t>(V) % 16 == 0;
}

size_t panel_tc_bytes(int64_t E, int32_t n_steps, int32_t nrhs) {
    return panel_plan(E, n_steps, nrhs).xf_bytes;
}
int panel_tc_max_slices() { return PN_MAX_Z; }

stb_status panel_tc_begin(int64_t E, int32_t n_steps, int32_t nrhs, void *xf, cudaStream_t s) {
    STB_CUDA(cudaMemsetAsync(xf, 0, panel_plan(E, n_steps, nrhs).xf_bytes, s));
    return STB_OK;
}

template <int N>
static stb_status panel_launch(const CUtensorMap &map, const CUtensorMap &mapA,
                               const PanelArgs &args, const PanelPlan &p, int n_z, cudaStream_t s) {
    using Sh = PanelShape<N>;
    const auto kern = k_toeplitz_panel<N>;
    STB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM));
    count_launch(s);
    kern<<<dim3((unsigned)p.row_tiles, 1, (unsigned)n_z), PN_THREADS, Sh::SMEM, s>>>(map, mapA, args);
    return check_launch("k_toeplitz_panel");
}

stb_status panel_tc(const float *V, int64_t E, int32_t n_steps, int32_t nrhs, const float *x,
                    int kp, int nb, void *xf, float *part, int *n_z_out, int32_t *status,
                    cudaStream_t s) {
    const PanelPlan p = panel_plan(E, n_steps, nrhs);
    __nv_bfloat16 *Xf = static_cast<__nv_bfloat16 *>(xf);
    stb_status st;
    {  // slices of the steps solved in the previous panel
        const int m_lo = std::max(0, kp - PN_PB), m_hi = kp;
        const size_t total = (size_t)(m_hi - m_lo) * nrhs * ((E + 1) / 2);
        if (total) {
            count_launch(s);
            k_panel_split_x<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
                x, (int)E, p.E_pad, n_steps, nrhs, p.rpad, p.rowsX, m_lo, m_hi, Xf);
            if ((st = check_launch("k_panel_split_x"))) return st;
        }
    }
    if (!panel_tc_blocks_ok(V, E))
        return fail(STB_ERR_INVALID_ARG, "panel product: E must be a multiple of 4, V 16-byte aligned");
    CUtensorMap map, mapA;
    if ((st = tc_make_map_2d(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Xf,
                             (uint64_t)PN_NS * p.rowsX, (uint64_t)p.E_pad, SP_KC, (uint32_t)p.N)))
        return st;
    // V as n_steps E rows of E FP32 columns; boxes of 128 rows x 32 columns
    if ((st = tc_make_map_2d(&mapA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, V,
                             (uint64_t)n_steps * E, (uint64_t)E, 32, SP_M)))
        return st;
    // blocks d = 1 .. kp + nb - 1, cut into at most PN_MAX_Z slices, about 16
    // waves of one CTA per SM: each CTA sums few blocks in its FP32 tensor
    // memory accumulator and the slices are added in FP64, which keeps the
    // FP32 rounding of the long sums near that of the SIMT march
    const int d_lo = 1, d_end = kp + nb;
    const int n_d = d_end - d_lo;
    const int64_t want = (16 * 152 + p.row_tiles - 1) / p.row_tiles;
    int n_z = (int)std::min<int64_t>(std::min<int64_t>(PN_MAX_Z, want), n_d);
    const int dr_len = (n_d + n_z - 1) / n_z;
    n_z = (n_d + dr_len - 1) / dr_len;
    *n_z_out = n_z;
    PanelArgs args{V, part, status, (int)E, nrhs, p.rpad, p.rowsX, p.n_chunks, kp, nb, d_lo, d_end,
                   dr_len};
    switch (p.N) {
    case 16: return panel_launch<16>(map, mapA, args, p, n_z, s);
    case 32: return panel_launch<32>(map, mapA, args, p, n_z, s);
    case 64: return panel_launch<64>(map, mapA, args, p, n_z, s);
    default: return fail(STB_ERR_INVALID_ARG, "panel product: at most 8 right-hand sides");
    }
}

}  // namespace stb
