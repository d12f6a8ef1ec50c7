// stb_mixed_math.h -- FP32 helpers shared by the mixed-precision assembly
// kernels: the MUFU exp2, the bracket psi of the double-layer antiderivative
// and the table loads from shared memory.
#pragma once
#include <cstdint>

namespace stb {

constexpr float ISQRTPI = 0.5641895835477563f;  // 1/sqrt(pi)

__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// psi(x) = erf(x)/2 - erf(x)/(4x^2) + exp(-x^2)/(2 sqrt(pi) x) (bracket of
// eq. dG); ix = 1/x
__device__ __forceinline__ float psi32(float x, float ix, float erfx, float ex) {
    if (x < 0.5f) {
        // (2/sqrt(pi)) sum_m (-1)^m x^{2m+1} / (m! (2m+1)(2m+3)), m <= 6
        float x2 = x * x;
        float p = 1.0f / (720.0f * 13.0f * 15.0f);          // m = 6
        p = fmaf(p, x2, -1.0f / (120.0f * 11.0f * 13.0f));  // m = 5
        p = fmaf(p, x2, 1.0f / (24.0f * 9.0f * 11.0f));     // m = 4
        p = fmaf(p, x2, -1.0f / (6.0f * 7.0f * 9.0f));      // m = 3
        p = fmaf(p, x2, 1.0f / (2.0f * 5.0f * 7.0f));       // m = 2
        p = fmaf(p, x2, -1.0f / (3.0f * 5.0f));             // m = 1
        p = fmaf(p, x2, 1.0f / 3.0f);                       // m = 0
        return 2.0f * ISQRTPI * x * p;
    }
    return 0.5f * erfx - 0.25f * erfx * ix * ix + 0.5f * ISQRTPI * ex * ix;
}

// 16-byte table load; SMEM: from shared memory, as a volatile access so that
// the compiler does not hoist a whole chunk of table entries into registers
// out of the quadrature-point loops.
template <bool SMEM>
__device__ __forceinline__ float4 ld_tab(const float *p) {
    if constexpr (SMEM) {
        float4 v;
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                     : "r"((uint32_t)__cvta_generic_to_shared(p)));
        return v;
    } else {
        return *reinterpret_cast<const float4 *>(p);
    }
}

}  // namespace stb
