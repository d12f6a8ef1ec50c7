// stb_grid.cuh -- grid-wide barrier of a cooperative launch, with a bounded
// wait, and the launch helper.  Used by the kernels that run a sequence of
// dependent phases (the time march of a panel, the blocked Cholesky) in one
// launch instead of one launch per phase.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "stb_internal.h"

namespace stb {

// Default limit of a grid barrier wait: 2 s.
constexpr uint64_t GRID_WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint64_t grid_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Barrier words in global memory: bar[0] arrivals, bar[1] generation,
// bar[2] abort flag.  bar[0] and bar[2] must be zero when the launch starts
// (grid_barrier_reset); every barrier leaves bar[0] at zero again.
//
// All CTAs of the launch must be resident at once (a cooperative launch of at
// most the occupancy limit).  Thread 0 of each CTA arrives with a device-scope
// atomic after a fence that publishes the CTA's writes; the last arrival
// resets the count and advances the generation, the others poll the
// generation.  A wait gives up after limit_ns (default GRID_WAIT_NS): it sets
// the abort flag and STB_ERR_TIMEOUT in *status, and every CTA then sees
// `false` from this or its next barrier and must return.  Data written by
// other CTAs before the barrier must be read with L1-bypassing loads
// (__ldcg) after it.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int32_t *status,
                                             uint64_t limit_ns = GRID_WAIT_NS) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1, *abort = bar + 2;
        const unsigned g = *gen;
        __threadfence();
        bool ok = true;
        if (atomicAdd(bar, 1u) + 1 == gridDim.x * gridDim.y * gridDim.z) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const uint64_t t0 = grid_ns();
            for (uint32_t i = 1; *gen == g; ++i) {
                if ((i & 63u) == 0) {
                    if (*abort) {
                        ok = false;
                        break;
                    }
                    if (grid_ns() - t0 > limit_ns) {
                        atomicExch(bar + 2, 1u);
                        atomicCAS(status, 0, STB_ERR_TIMEOUT);
                        ok = false;
                        break;
                    }
                }
            }
        }
        __threadfence();
        ok_s = ok && *abort == 0;
    }
    __syncthreads();
    return ok_s != 0;
}

// Zero the arrival count and the abort flag before a launch (stream-ordered).
inline cudaError_t grid_barrier_reset(unsigned *bar, cudaStream_t s) {
    return cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), s);
}

// Largest grid (a multiple of the SM count, at most `per_sm` CTAs per SM)
// whose CTAs can all be resident at once.
template <class K>
inline int coop_grid(K kern, int threads, size_t smem, int per_sm) {
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess)
        return 0;
    return sms * (occ < per_sm ? occ : per_sm);
}

// Cooperative launch (all CTAs co-resident), capturable into a CUDA graph.
template <class... KArgs, class... Args>
inline cudaError_t launch_coop(void (*kern)(KArgs...), unsigned grid, unsigned threads, size_t smem,
                               cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

}  // namespace stb
