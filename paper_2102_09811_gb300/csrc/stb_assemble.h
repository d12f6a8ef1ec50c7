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
// Gauss-Legendre per interval [kh, (k+1)h]: MIX_NG1 nodes on k = 1; the
// intervals k >= 2 are evaluated in chunks of MIX_CH blocks d0..d0+MIX_CH-1:
// chunk d0 evaluates the intervals k = d0..d0+MIX_CH-1, each once, with
// mixed_chunk_ng(d0) nodes; the falling side of interval k feeds block k,
// the rising side block k+1 (the last one carried into the next chunk).
// The count follows the Gauss error on one interval of the hat-weighted
// kernel tau^{-3/2} exp(-a/tau), tau = t/h, a = r^2/(4 alpha h): measured
// relative to the entry wherever the entry is at least 1e-4 of its r = 0
// value, 4 nodes stay below 8e-7 from k = 2 on, 3 nodes below 1e-8 from
// k = 16 on and 2 nodes below 2e-7 from k = 96 on.  A chunk takes the count
// of its first interval, k = d0.
constexpr int MIX_NG1 = 6;
constexpr int MIX_CH = 16;
__host__ __device__ inline int mixed_chunk_ng(int d0) { return d0 < 16 ? 4 : d0 < 96 ? 3 : 2; }
// Node table: interval k = 1 as MIX_NG1 float4 (b, cVr, cKr, 0) (only its
// rising side, block 2, is needed); then per chunk MIX_CH intervals of
// mixed_iv_floats(ng) floats: float4 (b_0..b_3, unused entries 0), then per
// node float4 (cVf, cKf, cVr, cKr).  b is the exp2 scale
// -log2(e)/(4 alpha delta); c* fold the Gauss weight, the hat weight (falling
// side: block k, rising side: block k+1) and (4 pi alpha delta)^{-3/2} (K:
// times 1/(2 delta)).  Intervals past k = n_steps-1 (the tail of the last
// chunk) have zero weights.
constexpr int MIX_K1 = 4 * MIX_NG1;
__host__ __device__ inline int mixed_iv_floats(int ng) { return 4 + 4 * ng; }
inline size_t mixed_node_floats(int n_steps) {
    size_t n = MIX_K1;
    for (int d0 = 2; d0 < n_steps; d0 += MIX_CH)
        n += (size_t)MIX_CH * mixed_iv_floats(mixed_chunk_ng(d0));
    return n;
}
void mixed_tables(const stb_params &p, std::vector<float> &rule, std::vector<float> &ss,
                  std::vector<float> &nodes);
// Workspace layout of one problem (ws = nullptr: sizes only, L.bytes).
AssemblyLayout assembly_layout(const Mesh &m, const stb_params &p, void *ws, size_t cap);
stb_status check_assembly_params(const stb_params *p);
// FP64 path set-up of one problem: tables, geometry, pair classification.
stb_status prepare_fp64(const Mesh &m, const stb_params &p, const AssemblyLayout &L,
                        int32_t *status, cudaStream_t s);
// Mixed path set-up of one problem: tables, geometry, pair classification.
stb_status prepare_mixed(const Mesh &m, const stb_params &p, const AssemblyLayout &L,
                         int32_t *status, cudaStream_t s);
// Mixed-precision K with piecewise-linear trial functions into FP32 K1
// [n_steps][E][n_nodes] (zeroed here, filled with atomics); coords: the
// regularised rules' coordinates (s1, s2, t1, t2) per class, as FP32, in
// the order of the difference-form rules.
// Mixed-precision D^2 of the separated pairs added into FP32 D [n_steps][N][N].
stb_status run_d2_regular_mixed(const Mesh &m, const stb_params &p, float *D,
                                const AssemblyLayout &L, cudaStream_t s);
// Mixed-precision D^2 of the touching pairs (coords as for K1 below).
stb_status run_d2_singular_mixed(const Mesh &m, const stb_params &p, float *D,
                                 const AssemblyLayout &L, const float *coords, cudaStream_t s);
// V (FP32) and f = (1/2 M_h + K_h) g without storing K (f zeroed by the caller).
stb_status run_vrhs_mixed(const Mesh &m, const stb_params &p, float *V, const double *gd,
                          int nrhs, double *f, const AssemblyLayout &L, cudaStream_t s);
stb_status run_assembly_k1_mixed(const Mesh &m, const stb_params &p, float *K1,
                                 const AssemblyLayout &L, const float *coords, cudaStream_t s);
stb_status run_assembly_mixed(const Mesh &m, const stb_params &p, void *V, void *K,
                              const AssemblyLayout &L, cudaStream_t s);

// Non-uniform grid, mixed precision (stb_nonuniform_mixed.cu): host tables
// of the closed-form records (NU_CF_FLOATS floats: target offset, target
// count << 1 | small-x form allowed, 1/(2 sqrt(alpha delta_max)), the K
// constant of zero differences; then per difference c, 1/c, pV, sigma),
// the Gauss nodes (float4 b, cV, cK, tag) and the target blocks; and the
// separated-pair launch (FP64 blocks, touching pairs left out).
constexpr int NU_CF_FLOATS = 20;
void nu_mixed_tables(const stb_params &p, const double *t, std::vector<float> &cf,
                     std::vector<float> &nodes, std::vector<int32_t> &targets);
stb_status run_nu_regular_mixed(const Mesh &m, const stb_params &p, const double *geo,
                                const float *mrule, const float *d_cf, int n_cf,
                                const float *d_nodes, int n_nodes, const int32_t *d_targets,
                                double *V, double *K, cudaStream_t s);
// touching pairs of the same path (FP32 difference-form rules mss, per class
// ss_n[cls] points)
stb_status run_nu_singular_mixed(const Mesh &m, const stb_params &p, const double *geo,
                                 const TouchPair *pairs, const float *mss, const int (&ss_n)[4],
                                 const float *d_cf, int n_cf, const float *d_nodes, int n_nodes,
                                 const int32_t *d_targets, double *V, double *K, cudaStream_t s);

// Batched mixed assembly (one persistent launch for all pair classes of all
// problems: the touching pairs first, then the separated pairs).  upload_batch copies
// the problems' descriptors for work items of `tile` columns (host memory,
// not capturable); launch_batch only launches (capturable).
struct BatchDesc;
size_t batch_desc_bytes(int n);
stb_status upload_batch(const Mesh *const *meshes, const stb_params *params,
                        const AssemblyLayout *layouts, float *const *V, float *const *K, int n,
                        BatchDesc *d_descs, int tile, cudaStream_t s);
stb_status launch_batch(const Mesh *const *meshes, const stb_params *params,
                        const AssemblyLayout *layouts, float *const *V, float *const *K, int n,
                        const BatchDesc *d_descs, unsigned long long *counter, int tile, int stride,
                        cudaStream_t s);

}  // namespace stb
