// stb_peaks.cu -- throughput probes of the arithmetic pipes the kernels are
// bound by (no counterpart in the paper; the denominators of the rooflines):
// FP64 FMA, FP32 FMA and the MUFU exp2, each as eight independent chains per
// thread over a bounded number of iterations, timed with CUDA events.
#include "stb_internal.h"

namespace stb {

template <class T>
__global__ void k_probe_fma(T *out, int iters, T a, T b) {
    T x0 = (T)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5,
      x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__device__ __forceinline__ float probe_ex2(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void k_probe_ex2(float *out, int iters) {
    float x0 = -0.001f * threadIdx.x, x1 = x0 - 0.1f, x2 = x0 - 0.2f, x3 = x0 - 0.3f,
          x4 = x0 - 0.4f, x5 = x0 - 0.5f, x6 = x0 - 0.6f, x7 = x0 - 0.7f;
    for (int i = 0; i < iters; ++i) {
        x0 = -probe_ex2(x0); x1 = -probe_ex2(x1); x2 = -probe_ex2(x2); x3 = -probe_ex2(x3);
        x4 = -probe_ex2(x4); x5 = -probe_ex2(x5); x6 = -probe_ex2(x6); x7 = -probe_ex2(x7);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

}  // namespace stb

using namespace stb;

// ops per second of one timed launch (after an untimed one)
template <class F>
static stb_status time_probe(F launch, double ops, cudaStream_t s, double *rate) {
    cudaEvent_t a, b;
    STB_CUDA(cudaEventCreate(&a));
    STB_CUDA(cudaEventCreate(&b));
    launch();
    STB_CUDA(cudaEventRecord(a, s));
    launch();
    STB_CUDA(cudaEventRecord(b, s));
    STB_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    STB_CUDA(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *rate = ops / (ms * 1e-3);
    return check_launch("probe");
}

extern "C" stb_status stb_measure_peaks(double *fp64_fma_per_s, double *fp32_fma_per_s,
                                        double *ex2_per_s, stb_stream stream) {
    if (!fp64_fma_per_s || !fp32_fma_per_s || !ex2_per_s)
        return fail(STB_ERR_INVALID_ARG, "outputs must be given");
    int dev = 0, sms = 0;
    STB_CUDA(cudaGetDevice(&dev));
    STB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = 4 * sms, threads = 256;
    void *buf = nullptr;
    STB_CUDA(cudaMalloc(&buf, sizeof(double) * blocks * threads));
    const double lanes = (double)blocks * threads * 8.0;
    const int it64 = 4000, it32 = 40000, itx = 8000;
    stb_status st = time_probe([&] {
        k_probe_fma<double><<<blocks, threads, 0, s>>>((double *)buf, it64, 0.999, 0.001);
    }, lanes * it64, s, fp64_fma_per_s);
    if (!st) st = time_probe([&] {
        k_probe_fma<float><<<blocks, threads, 0, s>>>((float *)buf, it32, 0.999f, 0.001f);
    }, lanes * it32, s, fp32_fma_per_s);
    if (!st) st = time_probe([&] {
        k_probe_ex2<<<blocks, threads, 0, s>>>((float *)buf, itx);
    }, lanes * itx, s, ex2_per_s);
    cudaFree(buf);
    return st;
}
