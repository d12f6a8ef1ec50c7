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
#include <cuda.h>

#include <mutex>

#include "stb_internal.h"
#include "stb_toeplitz_tc.h"

namespace stb {

constexpr int TC_M = 128, TC_NB = 64, TC_K = 32;  // rows, columns per box, K tile (128 bytes)
constexpr int TC_STAGES = 4;
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_A_BYTES = TC_M * TC_K * 4, TC_BOX_BYTES = TC_NB * TC_K * 4;
constexpr uint64_t TC_WAIT_NS = 2000000000ull;  // 2 s
constexpr uint32_t TC_WAIT_SPINS = 1u << 28;

template <int NBOX>
struct TcShape {
    static constexpr int N = TC_NB * NBOX;
    static constexpr uint32_t STAGE = TC_A_BYTES + NBOX * TC_BOX_BYTES;
    static constexpr size_t SMEM = TC_STAGES * (size_t)STAGE + 1024 /*align*/ + 256 /*barriers*/;
    // kind::tf32 instruction descriptor: D FP32, A and B TF32, both K-major, M = 128
    static constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) |
                                      ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase of the given parity; false (and the status set) if it
// has not completed within TC_WAIT_NS or TC_WAIT_SPINS polls.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int32_t *status) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1; i < TC_WAIT_SPINS; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 1023u) == 0 && global_ns() - t0 > TC_WAIT_NS) break;
    }
    atomicCAS(status, 0, STB_ERR_TIMEOUT);
    return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// Shared-memory matrix descriptor of a K-major operand written by TMA with
// the 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;            // leading-dimension offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride offset between 8-row groups
    d |= (uint64_t)1 << 46;            // descriptor version
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}
template <int NBOX>
__device__ __forceinline__ void umma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(TcShape<NBOX>::IDESC), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t v[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
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
            const uint64_t da = smem_desc(sa), db = smem_desc(sa + TC_A_BYTES);
#pragma unroll
            for (int k = 0; k < TC_K / 8; ++k)  // 8 TF32 = 32 bytes: +2 in the address field
                umma_tf32<NBOX>(tmem, da + 2 * k, db + 2 * k, (it > 0 || k > 0) ? 1u : 0u);
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

// 2-D FP32 row-major tensor [rows][cols], box of box_rows x 32 columns
static stb_status make_map(CUtensorMap *map, const void *base, uint64_t rows, uint64_t cols,
                           uint32_t box_rows) {
    EncodeTiledFn fn;
    stb_status st = encode_fn(&fn);
    if (st) return st;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 4};
    const cuuint32_t box[2] = {(cuuint32_t)TC_K, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult res =
        fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box,
           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (res != CUDA_SUCCESS)
        return fail(STB_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)res);
    return STB_OK;
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

}  // namespace stb
