// stb_toeplitz_tc.cu -- block-Toeplitz product (eq. V_mat) on the tcgen05
// tensor cores: FP32 blocks read as TF32, FP32 accumulation in tensor memory.
//
//   y_r^k = beta y_r^k + sum_{d=0}^{k} A^d x_r^{k-d}
//
// As one GEMM: Y (E x n_steps) = [A^0 ... A^{E_t-1}] (E x E_t E) times a
// Toeplitz-shifted copy of X whose column k in K-slice d is x^{k-d}.  With X
// stored padded, Xp[r][E_t + k][:] = x_r^k and zero rows before it, the
// 64-column B box of (block d, steps n0..n0+63) is the contiguous row window
// Xp[r][E_t + n0 - d .. +64): a plain 2-D TMA box, no gather.
//
// A CTA owns 128 rows of A, NBOX boxes of 64 columns (same n0, consecutive
// right-hand sides, or consecutive n0 of one right-hand side) and a slice of
// the blocks d.  Warp 0 issues TMA loads of 128x32 A and NBOX 64x32 B tiles
// (FP32, 128-byte swizzle) into a 4-stage ring, warp 1 issues tcgen05.mma
// (kind::tf32, M=128, N=64*NBOX, K=8; four per tile) into an FP32 accumulator
// in tensor memory, then all four warps read it back (tcgen05.ld) and store a
// partial slice; k_tc_reduce adds the slices in FP64.  Blocks d > n0 + 63 meet
// only the zero rows of Xp and are skipped.  Every mbarrier wait is bounded in
// time and iterations; an expired wait writes STB_ERR_TIMEOUT to the status.
#include <mutex>

#include "stb_tc.cuh"
#include "stb_toeplitz_tc.h"

namespace stb {

constexpr int TC_M = 128, TC_NB = 64, TC_K = 32;  // rows, columns per box, K tile (128 bytes)
constexpr int TC_STAGES = 4;
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_A_BYTES = TC_M * TC_K * 4, TC_BOX_BYTES = TC_NB * TC_K * 4;

template <int NBOX>
struct TcShape {
    static constexpr int N = TC_NB * NBOX;
    static constexpr uint32_t STAGE = TC_A_BYTES + NBOX * TC_BOX_BYTES;
    static constexpr size_t SMEM = TC_STAGES * (size_t)STAGE + 1024 /*align*/ + 256 /*barriers*/;
    static constexpr uint32_t IDESC = idesc_tf32(TC_M, N);
};

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int32_t *status) {
    return mbar_wait_bounded(bar, parity, status, nullptr, TC_WAIT_NS);
}

// Column box ct (0 <= ct < nrhs * n_tiles), ordered by n0 first so that the
// boxes of one CTA share n0 when there are several right-hand sides.
struct Box {
    int r, n0;
};
__device__ __forceinline__ Box box_of(int ct, int nrhs) {
    return Box{ct % nrhs, (ct / nrhs) * TC_NB};
}

template <int NBOX>
__global__ void __launch_bounds__(TC_THREADS)
k_toeplitz_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              int E, int n_steps, int nrhs, int n_ct, int dr_len, float *__restrict__ part,
              int32_t *__restrict__ status) {
    using Sh = TcShape<NBOX>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + TC_STAGES * Sh::STAGE);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * TC_STAGES + 1);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + TC_STAGES),
                   done = smem_u32(bars + 2 * TC_STAGES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const int m0 = blockIdx.x * TC_M;
    const int ct0 = blockIdx.y * NBOX;
    int n0_max = 0;
#pragma unroll
    for (int b = 0; b < NBOX; ++b)
        if (ct0 + b < n_ct) n0_max = max(n0_max, box_of(ct0 + b, nrhs).n0);
    const int d0 = blockIdx.z * dr_len;
    const int d1 = min(min(d0 + dr_len, n_steps), n0_max + TC_NB);
    if (d0 >= d1) return;  // only zero rows of Xp: k_tc_reduce never reads this slice
    const int kt_per_d = (E + TC_K - 1) / TC_K;
    const int n_iter = (d1 - d0) * kt_per_d;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {  // tensor memory: N FP32 columns x 128 lanes
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(Sh::N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {  // TMA producer
        int brow[NBOX];            // B row of each box at d = 0
#pragma unroll
        for (int b = 0; b < NBOX; ++b) {
            const Box bx = box_of(min(ct0 + b, n_ct - 1), nrhs);  // unused boxes repeat a valid one
            brow[b] = bx.r * 2 * n_steps + n_steps + bx.n0;
        }
        for (int it = 0; it < n_iter; ++it) {
            const int s = it % TC_STAGES;
            if (!mbar_wait(empty0 + 8 * s, ((it / TC_STAGES) & 1) ^ 1, status)) break;
            const int d = d0 + it / kt_per_d, j0 = (it % kt_per_d) * TC_K;
            const uint32_t sa = smem_u32(smem + s * Sh::STAGE);
            mbar_expect_tx(full0 + 8 * s, Sh::STAGE);
            tma_load_2d(sa, &mapA, j0, d * E + m0, full0 + 8 * s);
#pragma unroll
            for (int b = 0; b < NBOX; ++b)
                tma_load_2d(sa + TC_A_BYTES + b * TC_BOX_BYTES, &mapB, j0, brow[b] - d,
                            full0 + 8 * s);
        }
    } else if (warp == 1 && lane == 0) {  // MMA issuer
        for (int it = 0; it < n_iter; ++it) {
            const int s = it % TC_STAGES;
            if (!mbar_wait(full0 + 8 * s, (it / TC_STAGES) & 1, status)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = smem_u32(smem + s * Sh::STAGE);
            const uint64_t da = smem_desc_sw128(sa), db = smem_desc_sw128(sa + TC_A_BYTES);
#pragma unroll
            for (int k = 0; k < TC_K / 8; ++k)  // 8 TF32 = 32 bytes: +2 in the address field
                umma_tf32(tmem, da + 2 * k, db + 2 * k, Sh::IDESC, (it > 0 || k > 0) ? 1u : 0u);
            umma_commit(empty0 + 8 * s);  // the stage is free once these MMAs have read it
        }
        umma_commit(done);  // arrives when every MMA issued above has completed
    }
    __syncwarp();
    const bool ok = mbar_wait(done, 0, status);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {  // warp w reads TMEM lanes 32w..32w+31 = rows of the tile
        const int row = m0 + warp * 32 + lane;
        const size_t slice = (size_t)blockIdx.z * nrhs * n_steps * E;
#pragma unroll 1
        for (int c0 = 0; c0 < Sh::N; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            const int ct = ct0 + c0 / TC_NB;
            if (row < E && ct < n_ct) {
                const Box bx = box_of(ct, nrhs);
                float *pr = part + slice + (size_t)bx.r * n_steps * E;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int k = bx.n0 + c0 % TC_NB + i;
                    if (k < n_steps) pr[(size_t)k * E + row] = __uint_as_float(v[i]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 2) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Sh::N)
                     : "memory");
    }
}

// Xp[r][n_steps + k][j] = tf32(x_r^k[j]) (round to nearest), zero rows Xp[r][0..n_steps)
__global__ void k_pad_x(const double *__restrict__ x, int E, int n_steps, int nrhs,
                        float *__restrict__ xp) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)nrhs * 2 * n_steps * E) return;
    const int j = (int)(i % E);
    const size_t rowi = i / E;
    const int row = (int)(rowi % (2 * n_steps)), r = (int)(rowi / (2 * n_steps));
    float v = 0.f;
    if (row >= n_steps) {
        const float xf = (float)x[((size_t)r * n_steps + (row - n_steps)) * E + j];
        uint32_t t;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(xf));
        v = __uint_as_float(t);
    }
    xp[i] = v;
}

// y = beta y + the sum of the slices z that hold blocks d <= k (FP64)
__global__ void k_tc_reduce(const float *__restrict__ part, int E, int n_steps, int nrhs, int dr_len,
                            double beta, double *__restrict__ y) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)nrhs * n_steps * E;
    if (idx >= total) return;
    const int k = (int)((idx / E) % n_steps);
    double s = 0.0;
    for (int z = 0; z * dr_len <= k; ++z) s += (double)part[(size_t)z * total + idx];
    y[idx] = beta == 0.0 ? s : fma(beta, y[idx], s);
}

// ------------------------------------------------------------------ host ---
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static stb_status encode_fn(EncodeTiledFn *out) {
    static std::mutex mu;
    static EncodeTiledFn fn = nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                               cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
            return fail(STB_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    *out = fn;
    return STB_OK;
}

// 2-D row-major tensor [rows][cols] of elem_bytes-byte elements, box of
// box_rows x box_cols elements (box_cols * elem_bytes = 128: one swizzled row)
stb_status tc_make_map_2d(CUtensorMap *map, CUtensorMapDataType type, uint32_t elem_bytes,
                          const void *base, uint64_t rows, uint64_t cols, uint32_t box_cols,
                          uint32_t box_rows) {
    EncodeTiledFn fn;
    stb_status st = encode_fn(&fn);
    if (st) return st;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * elem_bytes};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult res =
        fn(map, type, 2, const_cast<void *>(base), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (res != CUDA_SUCCESS)
        return fail(STB_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)res);
    return STB_OK;
}

// 2-D FP32 row-major tensor [rows][cols], box of box_rows x 32 columns
static stb_status make_map(CUtensorMap *map, const void *base, uint64_t rows, uint64_t cols,
                           uint32_t box_rows) {
    return tc_make_map_2d(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, rows, cols, TC_K,
                          box_rows);
}

struct TcPlan {
    int nbox, n_ct, n_y, n_z, dr_len;
};

static TcPlan tc_plan(int64_t E, int n_steps, int nrhs) {
    TcPlan p;
    const int n_tiles = (n_steps + TC_NB - 1) / TC_NB;
    p.n_ct = n_tiles * nrhs;
    p.nbox = p.n_ct >= 4 ? 4 : p.n_ct >= 2 ? 2 : 1;
    p.n_y = (p.n_ct + p.nbox - 1) / p.nbox;
    const int64_t base = ((E + TC_M - 1) / TC_M) * p.n_y;  // CTAs per slice of blocks
    const int64_t want = 4 * 152 * (p.nbox == 1 ? 2 : 1);  // about four waves
    int64_t n_z = base >= want ? 1 : (want + base - 1) / base;
    if (n_z > n_steps) n_z = n_steps;
    p.dr_len = (int)((n_steps + n_z - 1) / n_z);
    p.n_z = (n_steps + p.dr_len - 1) / p.dr_len;
    return p;
}

size_t toeplitz_tc_bytes(int64_t E, int32_t n_steps, int32_t nrhs) {
    const TcPlan p = tc_plan(E, n_steps, nrhs);
    return align256((size_t)nrhs * 2 * n_steps * E * sizeof(float)) +
           align256((size_t)p.n_z * nrhs * n_steps * E * sizeof(float));
}

template <int NBOX>
static stb_status launch_tc(const CUtensorMap &mA, const CUtensorMap &mB, const TcPlan &p, int64_t E,
                            int n_steps, int nrhs, float *part, int32_t *status, cudaStream_t s) {
    using Sh = TcShape<NBOX>;
    STB_CUDA(cudaFuncSetAttribute(k_toeplitz_tc<NBOX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)Sh::SMEM));
    const dim3 grid((unsigned)((E + TC_M - 1) / TC_M), (unsigned)p.n_y, (unsigned)p.n_z);
    count_launch(s);
    k_toeplitz_tc<NBOX><<<grid, TC_THREADS, Sh::SMEM, s>>>(mA, mB, (int)E, n_steps, nrhs, p.n_ct,
                                                           p.dr_len, part, status);
    return check_launch("k_toeplitz_tc");
}

stb_status toeplitz_tc(const float *A, int64_t E, int32_t n_steps, int32_t nrhs, const double *x,
                       double beta, double *y, void *scratch, int32_t *status, cudaStream_t s) {
    if (E % 4 != 0) return fail(STB_ERR_INVALID_ARG, "the TF32 product needs E divisible by 4");
    if (reinterpret_cast<uintptr_t>(A) % 16 != 0)
        return fail(STB_ERR_INVALID_ARG, "the TF32 product needs 16-byte aligned blocks");
    const TcPlan p = tc_plan(E, n_steps, nrhs);
    float *xp = static_cast<float *>(scratch);
    float *part = reinterpret_cast<float *>(static_cast<char *>(scratch) +
                                            align256((size_t)nrhs * 2 * n_steps * E * sizeof(float)));
    const size_t nx = (size_t)nrhs * 2 * n_steps * E;
    count_launch(s);
    k_pad_x<<<(unsigned)((nx + 255) / 256), 256, 0, s>>>(x, (int)E, n_steps, nrhs, xp);
    stb_status st = check_launch("k_pad_x");
    if (st) return st;
    CUtensorMap mapA, mapB;
    if ((st = make_map(&mapA, A, (uint64_t)n_steps * E, (uint64_t)E, TC_M))) return st;
    if ((st = make_map(&mapB, xp, (uint64_t)nrhs * 2 * n_steps, (uint64_t)E, TC_NB))) return st;
    st = p.nbox == 4   ? launch_tc<4>(mapA, mapB, p, E, n_steps, nrhs, part, status, s)
         : p.nbox == 2 ? launch_tc<2>(mapA, mapB, p, E, n_steps, nrhs, part, status, s)
                       : launch_tc<1>(mapA, mapB, p, E, n_steps, nrhs, part, status, s);
    if (st) return st;
    const size_t total = (size_t)nrhs * n_steps * E;
    count_launch(s);
    k_tc_reduce<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(part, (int)E, n_steps, nrhs,
                                                                p.dr_len, beta, y);
    return check_launch("k_tc_reduce");
}

// One CTA: a bulk copy waited for with the bounded wait, then a bounded wait
// on a barrier nothing arrives on (unless `arrive`): the expiry path of every
// tensor-core kernel, without a fault.
__global__ void k_selftest_wait(const void *probe, uint64_t limit_ns, int arrive,
                                int32_t *status) {
    __shared__ __align__(128) unsigned char buf[256];
    __shared__ __align__(8) uint64_t bars[2];
    if (threadIdx.x != 0) return;
    const uint32_t b0 = smem_u32(&bars[0]), b1 = smem_u32(&bars[1]);
    mbar_init(b0, 1);
    mbar_init(b1, 1);
    mbar_init_fence();
    mbar_expect_tx(b0, sizeof buf);
    bulk_load(smem_u32(buf), probe, sizeof buf, b0);
    if (!mbar_wait_bounded(b0, 0, status, nullptr, TC_WAIT_NS)) return;  // the copy has landed
    if (arrive) mbar_arrive(b1);
    mbar_wait_bounded(b1, 0, status, nullptr, limit_ns);
}

}  // namespace stb

using namespace stb;

extern "C" stb_status stb_selftest_bounded_wait(const void *probe, int64_t limit_ns, int32_t arrive,
                                                void *ws, size_t ws_bytes, stb_stream stream) {
    if (!probe || reinterpret_cast<uintptr_t>(probe) % 16 != 0)
        return fail(STB_ERR_INVALID_ARG, "probe must be a 16-byte aligned device pointer");
    if (limit_ns < 1000 || limit_ns > 10000000000ll)
        return fail(STB_ERR_INVALID_ARG, "limit_ns must lie in [1000, 1e10]");
    stb_status st = check_workspace(ws, ws_bytes, 256);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    count_launch(s);
    k_selftest_wait<<<1, 32, 0, s>>>(probe, (uint64_t)limit_ns, arrive, status_word(ws));
    return check_launch("k_selftest_wait");
}

