// stb_internal.h -- internal declarations shared by the library's translation
// units (host + device).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstdint>
#include <vector>

#include "../../include/stbem.h"

namespace stb {

// ---------------------------------------------------------------- errors ----
stb_status fail(stb_status code, const char *fmt, ...);
stb_status cuda_fail(cudaError_t err, const char *what);
#define STB_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return stb::cuda_fail(e_, #call); \
    } while (0)

// Launch bookkeeping: every kernel launch of the library is preceded by
// count_launch(stream) and followed by check_launch(kernel name).  The pair
// counts the launch (stb_launch_count) and, while tracing is on, brackets it
// with CUDA events on its stream (stb_trace_*).
extern std::atomic<int64_t> g_launches;
void count_launch(cudaStream_t s);
stb_status check_launch(const char *what);

// ------------------------------------------------------------------ mesh ----
struct Mesh {
    int64_t n_nodes = 0, n_tris = 0, n_touch = 0;  // unordered touching pairs (a <= b)
    std::vector<double> nodes;                     // host copy [n_nodes][3]
    std::vector<int32_t> tris;                     // host copy [E][3]
    double *d_nodes = nullptr;                     // device copies
    int32_t *d_tris = nullptr;
};

// Per-triangle geometry record in device memory (16 doubles, 128 B).
// v0, v1, v2 vertices; n outward unit normal; area.
enum { GEO_V0 = 0, GEO_V1 = 3, GEO_V2 = 6, GEO_N = 9, GEO_AREA = 12, GEO_STRIDE = 16 };

// Pair classes (Sec. 3.1: separated pairs vs pairs sharing a vertex, an edge
// or the whole triangle).
enum { PAIR_DISJOINT = 0, PAIR_VERTEX = 1, PAIR_EDGE = 2, PAIR_IDENTICAL = 3 };

// One unordered touching pair a <= b.  `perm` packs the local vertex orders
// oa (bits 0..5) and ob (bits 6..11), two bits per position.
struct TouchPair {
    int32_t a, b, cls, perm;
};

// ------------------------------------------------------------ workspace ----
// Bump allocator over a caller workspace; the first 256 bytes hold the status
// word (int32) of the call.
struct Carve {
    char *base;
    size_t off, cap;
    explicit Carve(void *p, size_t c) : base(static_cast<char *>(p)), off(256), cap(c) {}
    template <class T> T *take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += n * sizeof(T);
        return p;
    }
    bool fits() const { return off <= cap; }
};
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
stb_status check_workspace(void *ws, size_t bytes, size_t need);
int32_t *status_word(void *ws);

// -------------------------------------------------------- quadrature (host) --
// Gauss-Legendre on [0,1] and Gauss-Jacobi (weight x on [0,1]) by the
// Golub-Welsch eigenvalue method.
void gauss_legendre01(int n, double *x, double *w);
void gauss_jacobi_x01(int n, double *x, double *w);
// Conical product rule on T = {0 <= s2 <= s1 <= 1}: q*q points (s1, s2, w).
void triangle_rule(int q, std::vector<double> &s1, std::vector<double> &s2,
                   std::vector<double> &w);
// Regularised rule of a touching class on T x T: points (s1, s2, t1, t2, w).
int ss_rule_size(int cls, int m);
void ss_rule(int cls, int m, std::vector<double> &s1, std::vector<double> &s2,
             std::vector<double> &t1, std::vector<double> &t2, std::vector<double> &w);
// The same rule in difference form, so that x - y keeps its relative accuracy
// as it shrinks (shared vertices first in both triangles, P_i, Q_i their
// vertices, A_i = P_i - P_{i-1}, B_i = Q_i - Q_{i-1}):
//   identical: (z1, z2, -, -),   x - y = -(z1 A1 + z2 A2),      z = t - s
//   edge     : (u, s2, t2, -),   x - y = -u A1 + s2 A2 - t2 B2,  u = t1 - s1
//   vertex   : (s1, s2, t1, t2), x - y = s1 A1 + s2 A2 - t1 B1 - t2 B2
void ss_rule_diff(int cls, int m, std::vector<double> &p0, std::vector<double> &p1,
                  std::vector<double> &p2, std::vector<double> &p3, std::vector<double> &w);

// ------------------------------------------------------- kernel launchers --
stb_status launch_geometry(const Mesh &m, double *geo, cudaStream_t s);
stb_status launch_classify(const Mesh &m, int32_t *row_count, int32_t *row_off,
                           TouchPair *pairs, int32_t *status, cudaStream_t s);

}  // namespace stb

struct stb_mesh {
    stb::Mesh m;
};
