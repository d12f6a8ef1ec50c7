// stb_heat.h -- the heat kernel G_alpha(r, tau) (Sec. 2) for the data and
// error kernels, FP64 or FP32 (mixed precision: exp2 on the MUFU pipe and a
// reciprocal square root); rr = |r|^2, zero for tau <= 0.
#pragma once
#include <cuda_runtime.h>

namespace stb {
template <class R> __device__ __forceinline__ R heat(R rr, R tau, R alpha);
template <> __device__ __forceinline__ double heat<double>(double rr, double tau, double alpha) {
    if (tau <= 0.0) return 0.0;
    const double s = 4.0 * 3.14159265358979323846 * alpha * tau;
    return exp(-rr / (4.0 * alpha * tau)) / (s * sqrt(s));
}
template <> __device__ __forceinline__ float heat<float>(float rr, float tau, float alpha) {
    if (tau <= 0.0f) return 0.0f;
    const float s = 4.0f * 3.14159265f * alpha * tau;
    float e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-rr / (4.0f * alpha * tau) * 1.44269504f));
    return e * rsqrtf(s * s * s);
}
}  // namespace stb
