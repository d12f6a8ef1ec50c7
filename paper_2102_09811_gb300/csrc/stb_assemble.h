// stb_assemble.h -- internal interface between the assembly driver and the
// FP64 / mixed-precision kernels.
#pragma once
#include <vector>

#include "stb_internal.h"

namespace stb {

struct AssemblyLayout {
    double *geo;
    int32_t *row_count, *row_off;
    TouchPair *pairs;
    double *rule, *ss, *levels;  // FP64 path: regular rule, regularised rules, level constants
    float *mrule, *mss, *mnodes; // mixed path: regular rule, difference-form rules, time nodes
    size_t ss_n[4];
    size_t bytes;
};

// Mixed path time quadrature of eq. V_d reduced to one variable,
//   V^d(r) = int_{(d-1)h}^{dh} (s-(d-1)h) G(r,s) ds + int_{dh}^{(d+1)h} ((d+1)h-s) G(r,s) ds,
// Gauss-Legendre per interval [kh, (k+1)h]: MIX_NG1 nodes on k = 1, MIX_NG on k >= 2.
constexpr int MIX_NG1 = 6;
constexpr int MIX_NG = 4;
// Node table: interval k = 1 as MIX_NG1 float4 (b, cVr, cKr, 0) (only its
// rising side, block 2, is needed); every interval k >= 2 as MIX_IV floats:
// float4 (b_0..b_3), then per node float4 (cVf, cKf, cVr, cKr).  b is the
// exp2 scale -log2(e)/(4 alpha delta); c* fold the Gauss weight, the hat
// weight (falling side: block k, rising side: block k+1) and (4 pi alpha
// delta)^{-3/2} (K: times 1/(2 delta)).
constexpr int MIX_K1 = 4 * MIX_NG1;
constexpr int MIX_IV = 4 + 4 * MIX_NG;
inline size_t mixed_node_floats(int n_steps) {
    return (size_t)MIX_K1 + (size_t)MIX_IV * (size_t)(n_steps > 2 ? n_steps - 2 : 0);
}
void mixed_tables(const stb_params &p, std::vector<float> &rule, std::vector<float> &ss,
                  std::vector<float> &nodes);
stb_status run_assembly_mixed(const Mesh &m, const stb_params &p, void *V, void *K,
                              const AssemblyLayout &L, cudaStream_t s);

}  // namespace stb
