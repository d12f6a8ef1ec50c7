// stb_assemble.cu -- triangle geometry, pair classification and the FP64
// assembly of the Toeplitz blocks V^d, K^d (Sec. 3.1-3.2, Sec. 5).
//
// Work decomposition (GB300):
//  * separated pairs: one thread per (test l, trial j) pair, a CTA covers 128
//    consecutive trial triangles of one test triangle, so every store of a
//    block entry V^d[l][j] is coalesced over j.  The time levels i_t = 1..E_t
//    are processed in chunks of CH levels whose spatial sums stay in
//    registers; the pair geometry (rho, 1/rho, r.n_y/rho) of a quadrature point
//    is recomputed once per chunk, so one heat-kernel evaluation costs one
//    erf + one exp shared by V and K.  After a chunk the second differences of
//    eq. vd / eq. V0 (and eq. K_d / eq. K0) are formed from a sliding window of
//    three level sums (Table deltad read as a gather: block d needs levels
//    d-1, d, d+1), so no atomics and no re-reads are needed.
//  * touching pairs (shared vertex / edge / identical): one CTA of 128 threads
//    per unordered pair a <= b; the threads split the m^4 x sub-domain points
//    of the regularised rule, reduce each level chunk through shuffles and
//    shared memory, and one thread writes V^d and K^d of both (a,b) and (b,a):
//    the rule is built once for the ordered pair, so V^d is symmetric.
#include <cmath>
#include <map>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <vector>

#include "stb_assemble.h"

namespace stb {

// --------------------------------------------------------------- geometry ---
__global__ void k_geometry(const double *__restrict__ nodes, const int32_t *__restrict__ tris,
                           int64_t E, double *__restrict__ geo) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    double v[9];
    for (int k = 0; k < 3; ++k) {
        int32_t i = tris[3 * e + k];
        v[3 * k] = nodes[3 * i];
        v[3 * k + 1] = nodes[3 * i + 1];
        v[3 * k + 2] = nodes[3 * i + 2];
    }
    double u0 = v[3] - v[0], u1 = v[4] - v[1], u2 = v[5] - v[2];
    double w0 = v[6] - v[0], w1 = v[7] - v[1], w2 = v[8] - v[2];
    double n0 = u1 * w2 - u2 * w1, n1 = u2 * w0 - u0 * w2, n2 = u0 * w1 - u1 * w0;
    double len = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
    double *g = geo + e * GEO_STRIDE;
    for (int k = 0; k < 9; ++k) g[k] = v[k];
    g[GEO_N] = n0 / len;
    g[GEO_N + 1] = n1 / len;
    g[GEO_N + 2] = n2 / len;
    g[GEO_AREA] = 0.5 * len;
}

stb_status launch_geometry(const Mesh &m, double *geo, cudaStream_t s) {
    int64_t E = m.n_tris;
    count_launch(s);
    k_geometry<<<(unsigned)((E + 255) / 256), 256, 0, s>>>(m.d_nodes, m.d_tris, E, geo);
    return check_launch("k_geometry");
}

// ---------------------------------------------------------- classification ---
// Local vertex orders of a touching pair (the same reading as the regularised
// rules assume): shared vertices first and in the same order in both
// triangles; an edge pair rotates a so that the shared edge is (v0, v1) in a's
// cyclic order; a vertex pair rotates both so the shared vertex is v0.
__device__ __forceinline__ void classify_pair(const int32_t ta[3], const int32_t tb[3], int &cls,
                                              int &perm) {
    int sa[3], n = 0;
    for (int i = 0; i < 3; ++i) {
        sa[i] = (ta[i] == tb[0]) | (ta[i] == tb[1]) | (ta[i] == tb[2]);
        n += sa[i];
    }
    int oa[3] = {0, 1, 2}, ob[3] = {0, 1, 2};
    if (n == 3) {
        cls = PAIR_IDENTICAL;
    } else if (n == 2) {
        cls = PAIR_EDGE;
        int k = (sa[0] && sa[1]) ? 0 : (sa[1] && sa[2]) ? 1 : 2;
        for (int i = 0; i < 3; ++i) oa[i] = (k + i) % 3;
        int used = 0;
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j)
                if (tb[j] == ta[oa[i]]) {
                    ob[i] = j;
                    used |= 1 << j;
                }
        ob[2] = (used & 1) == 0 ? 0 : (used & 2) == 0 ? 1 : 2;
    } else if (n == 1) {
        cls = PAIR_VERTEX;
        int ka = sa[0] ? 0 : sa[1] ? 1 : 2;
        int kb = tb[0] == ta[ka] ? 0 : tb[1] == ta[ka] ? 1 : 2;
        for (int i = 0; i < 3; ++i) {
            oa[i] = (ka + i) % 3;
            ob[i] = (kb + i) % 3;
        }
    } else {
        cls = PAIR_DISJOINT;
    }
    perm = oa[0] | (oa[1] << 2) | (oa[2] << 4) | (ob[0] << 6) | (ob[1] << 8) | (ob[2] << 10);
}

__device__ __forceinline__ bool touches(const int32_t ta[3], const int32_t tb[3]) {
    bool t = false;
    for (int i = 0; i < 3; ++i) t |= (ta[i] == tb[0]) | (ta[i] == tb[1]) | (ta[i] == tb[2]);
    return t;
}

// One warp per row a: count (pass 0) or emit (pass 1) the pairs (a, b >= a)
// that share a vertex, in increasing b.
__global__ void k_classify(const int32_t *__restrict__ tris, int64_t E, int pass,
                           int32_t *__restrict__ row_count, const int32_t *__restrict__ row_off,
                           TouchPair *__restrict__ out, int64_t capacity) {
    int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (a >= E) return;
    int32_t ta[3] = {tris[3 * a], tris[3 * a + 1], tris[3 * a + 2]};
    int32_t cnt = 0;
    int32_t base = pass ? row_off[a] : 0;
    for (int64_t b0 = a; b0 < E; b0 += 32) {
        int64_t b = b0 + lane;
        bool t = false;
        int32_t tb[3];
        if (b < E) {
            tb[0] = tris[3 * b];
            tb[1] = tris[3 * b + 1];
            tb[2] = tris[3 * b + 2];
            t = touches(ta, tb);
        }
        unsigned bal = __ballot_sync(0xffffffffu, t);
        if (pass && t) {
            int cls, perm;
            classify_pair(ta, tb, cls, perm);
            int pos = base + cnt + __popc(bal & ((1u << lane) - 1u));
            if (pos < capacity) out[pos] = TouchPair{(int32_t)a, (int32_t)b, cls, perm};
        }
        cnt += __popc(bal);
    }
    if (!pass && lane == 0) row_count[a] = cnt;
}

// Exclusive scan of the row counts (one CTA); checks the total against the
// host's count of touching pairs.
__global__ void k_scan_rows(const int32_t *__restrict__ cnt, int64_t E, int32_t *__restrict__ off,
                            int64_t expect_total, int32_t *__restrict__ status) {
    __shared__ int64_t part[1024];
    int t = threadIdx.x, nt = blockDim.x;
    int64_t chunk = (E + nt - 1) / nt, lo = t * chunk, hi = min(E, lo + chunk);
    int64_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += cnt[i];
    part[t] = s;
    __syncthreads();
    for (int d = 1; d < nt; d <<= 1) {
        int64_t v = t >= d ? part[t - d] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = part[t] - s;
    for (int64_t i = lo; i < hi; ++i) {
        off[i] = (int32_t)run;
        run += cnt[i];
    }
    if (t == nt - 1) {
        off[E] = (int32_t)part[t];
        if (part[t] != expect_total) atomicCAS(status, 0, STB_ERR_BAD_MESH);
    }
}

stb_status launch_classify(const Mesh &m, int32_t *row_count, int32_t *row_off, TouchPair *pairs,
                           int32_t *status, cudaStream_t s) {
    int64_t E = m.n_tris;
    unsigned blocks = (unsigned)((E * 32 + 255) / 256);
    count_launch(s);
    k_classify<<<blocks, 256, 0, s>>>(m.d_tris, E, 0, row_count, row_off, pairs, m.n_touch);
    stb_status st = check_launch("k_classify(count)");
    if (st) return st;
    count_launch(s);
    k_scan_rows<<<1, 1024, 0, s>>>(row_count, E, row_off, m.n_touch, status);
    if ((st = check_launch("k_scan_rows"))) return st;
    count_launch(s);
    k_classify<<<blocks, 256, 0, s>>>(m.d_tris, E, 1, row_count, row_off, pairs, m.n_touch);
    return check_launch("k_classify(fill)");
}

// ------------------------------------------------------- kernel evaluation ---
// Per-level constants (level i >= 1, delta = i h) of the closed forms
//   G^{dtau dt}(r, delta)      = A rho erf(x) + B_i/rho erf(x) + C_i exp(-x^2)   (eq. G_dtau_dt)
//   alpha dG^{dtau dt}/dn_y    = (r.n/rho) [ (D_i/rho^2 - A') erf(x) - E_i/rho exp(-x^2) ]  (eq. dG)
// with x = rho c_i, c_i = 1/(2 sqrt(alpha delta)), A = 1/(8 pi alpha^2),
// B_i = delta/(4 pi alpha), C_i = sqrt(delta)/(4 pi sqrt(pi alpha^3)),
// A' = 1/(8 pi alpha), D_i = delta/(4 pi), E_i = sqrt(delta)/(4 pi sqrt(pi alpha)).
// For x < 1/2 the bracket of eq. dG cancels; it is evaluated as
//   alpha dG^{dtau dt}/dn_y = -(r.n/rho) psi(x) / (4 pi alpha),
//   psi(x) = (2/sqrt(pi)) sum_m (-1)^m x^{2m+1} / (m! (2m+1)(2m+3)).
// Level 0 uses the delta -> 0 limits of Sec. 3.1-3.2: A rho and -A' r.n/rho,
// and the delta = 0 integrands 1/(4 pi alpha rho) and r.n/(4 pi rho^3).
enum { LV_C = 0, LV_B, LV_CC, LV_D, LV_E, LV_STRIDE = 8 };
struct Globals {
    double A, Ap, F, Fs, h;  // F = 1/(4 pi alpha), Fs = 1/(4 pi)
};

__constant__ double c_psi[12];  // (2/sqrt(pi)) (-1)^m / (m! (2m+1)(2m+3))

static void upload_psi_coeffs(cudaStream_t s) {
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && done[dev]) return;
    double c[12];
    double fact = 1.0;
    for (int m = 0; m < 12; ++m) {
        if (m > 0) fact *= m;
        c[m] = (m % 2 ? -1.0 : 1.0) * 1.1283791670955126 / (fact * (2.0 * m + 1.0) * (2.0 * m + 3.0));
    }
    cudaMemcpyToSymbol(c_psi, c, sizeof c);
    if (dev < 64) done[dev] = true;
}

__device__ __forceinline__ double psi_series(double x) {
    double x2 = x * x, p = c_psi[11];
#pragma unroll
    for (int m = 10; m >= 0; --m) p = fma(p, x2, c_psi[m]);
    return p * x;
}

// V and K-factor at one level: V = G^{dtau dt}, Kf such that
// alpha dG^{dtau dt}/dn_y = (r.n/rho) * Kf.
__device__ __forceinline__ void eval_level(double rho, double irho, const double *lv,
                                           const Globals &g, double &v, double &kf) {
    double x = rho * lv[LV_C];
    double f = erf(x);
    double e = exp(-x * x);
    v = fma(fma(g.A, rho, lv[LV_B] * irho), f, lv[LV_CC] * e);
    if (x >= 0.5) {
        kf = fma(fma(lv[LV_D], irho * irho, -g.Ap), f, -lv[LV_E] * irho * e);
    } else {
        kf = -g.F * psi_series(x);
    }
}

template <class T> __device__ __forceinline__ void store(T *p, double v);
template <> __device__ __forceinline__ void store<double>(double *p, double v) { *p = v; }
template <> __device__ __forceinline__ void store<float>(float *p, double v) { *p = (float)v; }

// ------------------------------------------------- separated pairs, FP64 ---
constexpr int REG_THREADS = 128;
constexpr int MAX_RULE = 256;       // q <= 16
constexpr int MAX_LEVELS = 2049;    // n_steps <= 2048 (level table in smem)

template <int CH, class OutT>
__global__ void __launch_bounds__(REG_THREADS)
k_regular_f64(const double *__restrict__ geo, const int32_t *__restrict__ tris, int E,
              const double *__restrict__ rule, int nq, const double *__restrict__ levels,
              int n_steps, Globals g, OutT *__restrict__ V, OutT *__restrict__ K) {
    extern __shared__ double sm[];
    double *xa = sm;                   // [nq][4]: x_a (3) and w_a
    double *lv = sm + 4 * MAX_RULE;    // [n_steps+1][LV_STRIDE]
    const int l = blockIdx.y;
    const int j = blockIdx.x * REG_THREADS + threadIdx.x;
    const double *gl = geo + (size_t)l * GEO_STRIDE;
    for (int a = threadIdx.x; a < nq; a += REG_THREADS) {
        double s1 = rule[3 * a], s2 = rule[3 * a + 1];
        for (int c = 0; c < 3; ++c)
            xa[4 * a + c] = gl[GEO_V0 + c] + s1 * (gl[GEO_V1 + c] - gl[GEO_V0 + c]) +
                            s2 * (gl[GEO_V2 + c] - gl[GEO_V1 + c]);
        xa[4 * a + 3] = rule[3 * a + 2];
    }
    for (int i = threadIdx.x; i < (n_steps + 1) * LV_STRIDE; i += REG_THREADS) lv[i] = levels[i];
    __syncthreads();
    if (j >= E) return;
    const int32_t tl[3] = {tris[3 * l], tris[3 * l + 1], tris[3 * l + 2]};
    const int32_t tj[3] = {tris[3 * j], tris[3 * j + 1], tris[3 * j + 2]};
    if (touches(tl, tj)) return;  // written by the regularised-rule kernel

    const double *gj = geo + (size_t)j * GEO_STRIDE;
    double P0[3], e1[3], e2[3], n[3];
    for (int c = 0; c < 3; ++c) {
        P0[c] = gj[GEO_V0 + c];
        e1[c] = gj[GEO_V1 + c] - gj[GEO_V0 + c];
        e2[c] = gj[GEO_V2 + c] - gj[GEO_V1 + c];
        n[c] = gj[GEO_N + c];
    }
    const double scale = 4.0 * gl[GEO_AREA] * gj[GEO_AREA];
    const size_t EE = (size_t)E * E, ij = (size_t)l * E + j;

    // level 0: delta -> 0 limits and the delta = 0 singular integrands
    double s0v = 0, s0k = 0, ssv = 0, ssk = 0;
    for (int b = 0; b < nq; ++b) {
        double t1 = rule[3 * b], t2 = rule[3 * b + 1], wb = rule[3 * b + 2];
        double y0 = P0[0] + t1 * e1[0] + t2 * e2[0];
        double y1 = P0[1] + t1 * e1[1] + t2 * e2[1];
        double y2 = P0[2] + t1 * e1[2] + t2 * e2[2];
        for (int a = 0; a < nq; ++a) {
            double r0 = xa[4 * a] - y0, r1 = xa[4 * a + 1] - y1, r2 = xa[4 * a + 2] - y2;
            double rr = r0 * r0 + r1 * r1 + r2 * r2;
            double irho = rsqrt(rr), rho = rr * irho;
            double rnr = (r0 * n[0] + r1 * n[1] + r2 * n[2]) * irho;
            double w = xa[4 * a + 3] * wb;
            s0v = fma(w, g.A * rho, s0v);
            s0k = fma(w, -g.Ap * rnr, s0k);
            ssv = fma(w, g.F * irho, ssv);
            ssk = fma(w, g.Fs * rnr * irho * irho, ssk);
        }
    }
    double pv2 = 0, pk2 = 0;                   // S_{i-2}
    double pv1 = scale * s0v, pk1 = scale * s0k;  // S_{i-1}
    const double sv_sing = scale * ssv, sk_sing = scale * ssk;

    for (int c0 = 1; c0 <= n_steps; c0 += CH) {
        double sv[CH], sk[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) sv[u] = sk[u] = 0.0;
        for (int b = 0; b < nq; ++b) {
            double t1 = rule[3 * b], t2 = rule[3 * b + 1], wb = rule[3 * b + 2];
            double y0 = P0[0] + t1 * e1[0] + t2 * e2[0];
            double y1 = P0[1] + t1 * e1[1] + t2 * e2[1];
            double y2 = P0[2] + t1 * e1[2] + t2 * e2[2];
            for (int a = 0; a < nq; ++a) {
                double r0 = xa[4 * a] - y0, r1 = xa[4 * a + 1] - y1, r2 = xa[4 * a + 2] - y2;
                double rr = r0 * r0 + r1 * r1 + r2 * r2;
                double irho = rsqrt(rr), rho = rr * irho;
                double rnr = (r0 * n[0] + r1 * n[1] + r2 * n[2]) * irho;
                double w = xa[4 * a + 3] * wb, wk = w * rnr;
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    if (c0 + u <= n_steps) {
                        double v, kf;
                        eval_level(rho, irho, lv + (c0 + u) * LV_STRIDE, g, v, kf);
                        sv[u] = fma(w, v, sv[u]);
                        sk[u] = fma(wk, kf, sk[u]);
                    }
                }
            }
        }
        // second differences: level i = c0 + u completes block d = i - 1
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            int i = c0 + u;
            if (i <= n_steps) {
                double cv = scale * sv[u], ck = scale * sk[u];
                double bv, bk;
                if (i == 1) {  // eq. V0 / eq. K0
                    bv = g.h * sv_sing - cv + pv1;
                    bk = g.h * sk_sing - ck + pk1;
                } else {       // eq. vd / eq. K_d for d = i - 1
                    bv = 2.0 * pv1 - cv - pv2;
                    bk = 2.0 * pk1 - ck - pk2;
                }
                store(V + (size_t)(i - 1) * EE + ij, bv);
                if (K) store(K + (size_t)(i - 1) * EE + ij, bk);
                pv2 = pv1; pk2 = pk1;
                pv1 = cv;  pk1 = ck;
            }
        }
    }
}

// ------------------------------------------------- touching pairs, FP64 ---
constexpr int SS_THREADS = 128;

struct SSTables {
    const double *s1[4], *s2[4], *t1[4], *t2[4], *w[4];
    int n[4];
};

template <int CH, class OutT>
__global__ void __launch_bounds__(SS_THREADS)
k_singular_f64(const double *__restrict__ geo, const TouchPair *__restrict__ pairs, int E,
               SSTables tab, const double *__restrict__ levels, int n_steps, Globals g,
               OutT *__restrict__ V, OutT *__restrict__ K) {
    __shared__ double red[SS_THREADS / 32][3 * CH + 8];
    __shared__ double fin[3 * CH + 8];
    const TouchPair P = pairs[blockIdx.x];
    const int a = P.a, b = P.b, cls = P.cls;
    // slots are pre-filled with -1; a slot the classification did not write
    // (a count mismatch, reported through the status word) is skipped
    if (a < 0 || b < a || b >= E || cls < PAIR_VERTEX || cls > PAIR_IDENTICAL) return;
    const double *ga = geo + (size_t)a * GEO_STRIDE, *gb = geo + (size_t)b * GEO_STRIDE;
    double A0[3], A1[3], A2[3], B0[3], B1[3], B2[3], na[3], nb[3];
    {
        int oa0 = P.perm & 3, oa1 = (P.perm >> 2) & 3, oa2 = (P.perm >> 4) & 3;
        int ob0 = (P.perm >> 6) & 3, ob1 = (P.perm >> 8) & 3, ob2 = (P.perm >> 10) & 3;
        for (int c = 0; c < 3; ++c) {
            A0[c] = ga[3 * oa0 + c];
            A1[c] = ga[3 * oa1 + c] - ga[3 * oa0 + c];
            A2[c] = ga[3 * oa2 + c] - ga[3 * oa1 + c];
            B0[c] = gb[3 * ob0 + c];
            B1[c] = gb[3 * ob1 + c] - gb[3 * ob0 + c];
            B2[c] = gb[3 * ob2 + c] - gb[3 * ob1 + c];
            na[c] = ga[GEO_N + c];
            nb[c] = gb[GEO_N + c];
        }
    }
    const double scale = 4.0 * ga[GEO_AREA] * gb[GEO_AREA];
    const bool ident = cls == PAIR_IDENTICAL;
    const int npt = tab.n[cls];
    const double *S1 = tab.s1[cls], *S2 = tab.s2[cls], *T1 = tab.t1[cls], *T2 = tab.t2[cls],
                 *W = tab.w[cls];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t EE = (size_t)E * E, iab = (size_t)a * E + b, iba = (size_t)b * E + a;

    // point p: x on a, y on b; entry (a,b): r = x - y, n_b; entry (b,a): r' = -r, n_a
    auto point = [&](int p, double &rho, double &irho, double &rab, double &rba, double &w) {
        double s1 = S1[p], s2 = S2[p], t1 = T1[p], t2 = T2[p];
        double r[3];
        for (int c = 0; c < 3; ++c)
            r[c] = (A0[c] + s1 * A1[c] + s2 * A2[c]) - (B0[c] + t1 * B1[c] + t2 * B2[c]);
        double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        irho = rsqrt(rr);
        rho = rr * irho;
        rab = (r[0] * nb[0] + r[1] * nb[1] + r[2] * nb[2]) * irho;
        rba = -(r[0] * na[0] + r[1] * na[1] + r[2] * na[2]) * irho;
        w = W[p];
    };
    auto reduce = [&](double *vals, int nv) {
        for (int k = 0; k < nv; ++k) {
            double v = vals[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < nv) {
            double s = 0.0;
            for (int wi = 0; wi < SS_THREADS / 32; ++wi) s += red[wi][threadIdx.x];
            fin[threadIdx.x] = scale * s;
        }
        __syncthreads();
    };

    // level 0 and delta = 0 integrands
    double z[6] = {0, 0, 0, 0, 0, 0};
    for (int p = threadIdx.x; p < npt; p += SS_THREADS) {
        double rho, irho, rab, rba, w;
        point(p, rho, irho, rab, rba, w);
        z[0] = fma(w, g.A * rho, z[0]);
        z[1] = fma(w, -g.Ap * rab, z[1]);
        z[2] = fma(w, -g.Ap * rba, z[2]);
        z[3] = fma(w, g.F * irho, z[3]);
        z[4] = fma(w, g.Fs * rab * irho * irho, z[4]);
        z[5] = fma(w, g.Fs * rba * irho * irho, z[5]);
    }
    reduce(z, 6);
    // sliding window (only thread 0 uses it)
    double pv2 = 0, pa2 = 0, pb2 = 0, pv1 = fin[0], pa1 = fin[1], pb1 = fin[2];
    const double sv_s = fin[3], sa_s = fin[4], sb_s = fin[5];
    __syncthreads();

    for (int c0 = 1; c0 <= n_steps; c0 += CH) {
        double acc[3 * CH];
#pragma unroll
        for (int k = 0; k < 3 * CH; ++k) acc[k] = 0.0;
        for (int p = threadIdx.x; p < npt; p += SS_THREADS) {
            double rho, irho, rab, rba, w;
            point(p, rho, irho, rab, rba, w);
            double wa = w * rab, wb = w * rba;
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                if (c0 + u <= n_steps) {
                    double v, kf;
                    eval_level(rho, irho, levels + (c0 + u) * LV_STRIDE, g, v, kf);
                    acc[u] = fma(w, v, acc[u]);
                    acc[CH + u] = fma(wa, kf, acc[CH + u]);
                    acc[2 * CH + u] = fma(wb, kf, acc[2 * CH + u]);
                }
            }
        }
        reduce(acc, 3 * CH);
        if (threadIdx.x == 0) {
            for (int u = 0; u < CH; ++u) {
                int i = c0 + u;
                if (i > n_steps) break;
                double cv = fin[u], ca = fin[CH + u], cb = fin[2 * CH + u];
                double bv, ba, bb;
                if (i == 1) {
                    bv = g.h * sv_s - cv + pv1;
                    ba = g.h * sa_s - ca + pa1;
                    bb = g.h * sb_s - cb + pb1;
                } else {
                    bv = 2.0 * pv1 - cv - pv2;
                    ba = 2.0 * pa1 - ca - pa2;
                    bb = 2.0 * pb1 - cb - pb2;
                }
                size_t off = (size_t)(i - 1) * EE;
                store(V + off + iab, bv);
                if (!ident) store(V + off + iba, bv);
                if (K) {
                    // flat triangles: r . n_y vanishes on an identical pair
                    store(K + off + iab, ident ? 0.0 : ba);
                    if (!ident) store(K + off + iba, bb);
                }
                pv2 = pv1; pa2 = pa1; pb2 = pb1;
                pv1 = cv;  pa1 = ca;  pb1 = cb;
            }
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------- driver ---
AssemblyLayout assembly_layout(const Mesh &m, const stb_params &p, void *ws, size_t cap) {
    Carve c(ws, cap);
    AssemblyLayout L{};
    L.geo = c.take<double>((size_t)m.n_tris * GEO_STRIDE);
    L.row_count = c.take<int32_t>(m.n_tris);
    L.row_off = c.take<int32_t>(m.n_tris + 1);
    L.pairs = c.take<TouchPair>(m.n_touch > 0 ? m.n_touch : 1);
    size_t tot = 0;
    for (int cls = 1; cls <= 3; ++cls) {
        L.ss_n[cls] = ss_rule_size(cls, p.quad_singular);
        tot += 5 * L.ss_n[cls];
    }
    // one contiguous table region (uploaded with one copy)
    if (p.precision == STB_PREC_FP64) {
        L.rule = c.take<double>(3 * (size_t)p.quad_regular * p.quad_regular);
        L.ss = c.take<double>(tot);
        L.levels = c.take<double>((size_t)(p.n_steps + 1) * LV_STRIDE);
    } else {
        L.mrule = c.take<float>(4 * (size_t)p.quad_regular * p.quad_regular);
        L.mss = c.take<float>(tot);
        L.mnodes = c.take<float>(mixed_node_floats(p.n_steps));
    }
    L.bytes = c.off;
    return L;
}

stb_status check_assembly_params(const stb_params *p) {
    if (!p) return fail(STB_ERR_INVALID_ARG, "params is NULL");
    if (!(p->alpha > 0.0) || !(p->T > 0.0) || !std::isfinite(p->alpha) || !std::isfinite(p->T))
        return fail(STB_ERR_INVALID_ARG, "alpha and T must be positive and finite");
    if (p->n_steps < 1 || p->n_steps > MAX_LEVELS - 1)
        return fail(STB_ERR_INVALID_ARG, "n_steps must be in [1, %d]", MAX_LEVELS - 1);
    if (p->quad_regular < 1 || p->quad_regular > 16)
        return fail(STB_ERR_INVALID_ARG, "quad_regular must be in [1, 16]");
    if (p->quad_singular < 1 || p->quad_singular > 12)
        return fail(STB_ERR_INVALID_ARG, "quad_singular must be in [1, 12]");
    if (p->precision != STB_PREC_FP64 && p->precision != STB_PREC_MIXED)
        return fail(STB_ERR_INVALID_ARG, "precision must be STB_PREC_FP64 or STB_PREC_MIXED");
    if (p->precision == STB_PREC_MIXED && p->n_steps > 1024)
        return fail(STB_ERR_INVALID_ARG, "mixed precision supports n_steps <= 1024");
    if (p->storage != STB_STORE_F64 && p->storage != STB_STORE_F32)
        return fail(STB_ERR_INVALID_ARG, "storage must be STB_STORE_F64 or STB_STORE_F32");
    if (p->flags & ~(STB_FLAG_NO_SYNC | STB_FLAG_REFINE(15)))
        return fail(STB_ERR_INVALID_ARG, "unknown flags");
    return STB_OK;
}

static Globals make_globals(const stb_params &p) {
    const double pi = 3.14159265358979323846;
    Globals g;
    g.A = 1.0 / (8.0 * pi * p.alpha * p.alpha);
    g.Ap = 1.0 / (8.0 * pi * p.alpha);
    g.F = 1.0 / (4.0 * pi * p.alpha);
    g.Fs = 1.0 / (4.0 * pi);
    g.h = p.T / p.n_steps;
    return g;
}

// ---------------------------------------- piecewise-linear trial space ---
// K_h with nodal hat trial functions (Sec. 3.2): the K sums of a pair
// weighted by the barycentric coordinates of the trial point, their second
// differences per vertex, added to K1[d][l][node] (several trial triangles
// share a node, so the blocks are accumulated with atomics and must start
// at zero).
__device__ __forceinline__ void atomic_add_out(double *p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_out(float *p, double v) { atomicAdd(p, (float)v); }

template <int CH, class OutT>
__global__ void __launch_bounds__(REG_THREADS)
k_regular_k1_f64(const double *__restrict__ geo, const int32_t *__restrict__ tris, int E, int N,
                 const double *__restrict__ rule, int nq, const double *__restrict__ levels,
                 int n_steps, Globals g, OutT *__restrict__ K1) {
    extern __shared__ double sm[];
    double *xa = sm;                   // [nq][4]: x_a (3) and w_a
    double *lv = sm + 4 * MAX_RULE;    // [n_steps+1][LV_STRIDE]
    const int l = blockIdx.y;
    const int j = blockIdx.x * REG_THREADS + threadIdx.x;
    const double *gl = geo + (size_t)l * GEO_STRIDE;
    for (int a = threadIdx.x; a < nq; a += REG_THREADS) {
        double s1 = rule[3 * a], s2 = rule[3 * a + 1];
        for (int c = 0; c < 3; ++c)
            xa[4 * a + c] = gl[GEO_V0 + c] + s1 * (gl[GEO_V1 + c] - gl[GEO_V0 + c]) +
                            s2 * (gl[GEO_V2 + c] - gl[GEO_V1 + c]);
        xa[4 * a + 3] = rule[3 * a + 2];
    }
    for (int i = threadIdx.x; i < (n_steps + 1) * LV_STRIDE; i += REG_THREADS) lv[i] = levels[i];
    __syncthreads();
    if (j >= E) return;
    const int32_t tl[3] = {tris[3 * l], tris[3 * l + 1], tris[3 * l + 2]};
    const int32_t tj[3] = {tris[3 * j], tris[3 * j + 1], tris[3 * j + 2]};
    if (touches(tl, tj)) return;  // the regularised-rule kernel

    const double *gj = geo + (size_t)j * GEO_STRIDE;
    double P0[3], e1[3], e2[3], n[3];
    for (int c = 0; c < 3; ++c) {
        P0[c] = gj[GEO_V0 + c];
        e1[c] = gj[GEO_V1 + c] - gj[GEO_V0 + c];
        e2[c] = gj[GEO_V2 + c] - gj[GEO_V1 + c];
        n[c] = gj[GEO_N + c];
    }
    const double scale = 4.0 * gl[GEO_AREA] * gj[GEO_AREA];
    const size_t EN = (size_t)E * N;
    OutT *row = K1 + (size_t)l * N;

    // level 0 (delta -> 0 limit) and the delta = 0 singular integrand
    double s0[3] = {0, 0, 0}, ss[3] = {0, 0, 0};
    for (int b = 0; b < nq; ++b) {
        double t1 = rule[3 * b], t2 = rule[3 * b + 1], wb = rule[3 * b + 2];
        const double lam[3] = {1.0 - t1, t1 - t2, t2};
        double y0 = P0[0] + t1 * e1[0] + t2 * e2[0];
        double y1 = P0[1] + t1 * e1[1] + t2 * e2[1];
        double y2 = P0[2] + t1 * e1[2] + t2 * e2[2];
        for (int a = 0; a < nq; ++a) {
            double r0 = xa[4 * a] - y0, r1 = xa[4 * a + 1] - y1, r2 = xa[4 * a + 2] - y2;
            double rr = r0 * r0 + r1 * r1 + r2 * r2;
            double irho = rsqrt(rr);
            double rnr = (r0 * n[0] + r1 * n[1] + r2 * n[2]) * irho;
            double w = xa[4 * a + 3] * wb;
            double k0 = w * (-g.Ap * rnr), ks = w * g.Fs * rnr * irho * irho;
            for (int v = 0; v < 3; ++v) {
                s0[v] = fma(lam[v], k0, s0[v]);
                ss[v] = fma(lam[v], ks, ss[v]);
            }
        }
    }
    double p2[3], p1[3], sing[3];
    for (int v = 0; v < 3; ++v) {
        p2[v] = 0.0;
        p1[v] = scale * s0[v];
        sing[v] = scale * ss[v];
    }

    for (int c0 = 1; c0 <= n_steps; c0 += CH) {
        double sk[3][CH];
#pragma unroll
        for (int v = 0; v < 3; ++v)
#pragma unroll
            for (int u = 0; u < CH; ++u) sk[v][u] = 0.0;
        for (int b = 0; b < nq; ++b) {
            double t1 = rule[3 * b], t2 = rule[3 * b + 1], wb = rule[3 * b + 2];
            const double lam[3] = {1.0 - t1, t1 - t2, t2};
            double y0 = P0[0] + t1 * e1[0] + t2 * e2[0];
            double y1 = P0[1] + t1 * e1[1] + t2 * e2[1];
            double y2 = P0[2] + t1 * e1[2] + t2 * e2[2];
            for (int a = 0; a < nq; ++a) {
                double r0 = xa[4 * a] - y0, r1 = xa[4 * a + 1] - y1, r2 = xa[4 * a + 2] - y2;
                double rr = r0 * r0 + r1 * r1 + r2 * r2;
                double irho = rsqrt(rr), rho = rr * irho;
                double rnr = (r0 * n[0] + r1 * n[1] + r2 * n[2]) * irho;
                double wk = xa[4 * a + 3] * wb * rnr;
                const double wl[3] = {wk * lam[0], wk * lam[1], wk * lam[2]};
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    if (c0 + u <= n_steps) {
                        double v, kf;
                        eval_level(rho, irho, lv + (c0 + u) * LV_STRIDE, g, v, kf);
#pragma unroll
                        for (int q = 0; q < 3; ++q) sk[q][u] = fma(wl[q], kf, sk[q][u]);
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            int i = c0 + u;
            if (i <= n_steps) {
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    double c = scale * sk[v][u];
                    double bk = i == 1 ? g.h * sing[v] - c + p1[v]      // eq. K0
                                       : 2.0 * p1[v] - c - p2[v];      // eq. K_d, d = i - 1
                    atomic_add_out(row + (size_t)(i - 1) * EN + tj[v], bk);
                    p2[v] = p1[v];
                    p1[v] = c;
                }
            }
        }
    }
}

// Touching pairs: one CTA per unordered pair (a, b); entry (a, b) has its
// trial points on b (coordinates t1, t2 in b's rotated vertex order), entry
// (b, a) on a.  Identical pairs contribute nothing (r . n_y = 0).
template <int CH, class OutT>
__global__ void __launch_bounds__(SS_THREADS)
k_singular_k1_f64(const double *__restrict__ geo, const int32_t *__restrict__ tris,
                  const TouchPair *__restrict__ pairs, int E, int N, SSTables tab,
                  const double *__restrict__ levels, int n_steps, Globals g,
                  OutT *__restrict__ K1) {
    __shared__ double red[SS_THREADS / 32][6 * CH + 12];
    __shared__ double fin[6 * CH + 12];
    const TouchPair P = pairs[blockIdx.x];
    const int a = P.a, b = P.b, cls = P.cls;
    if (a < 0 || b < a || b >= E || cls < PAIR_VERTEX || cls >= PAIR_IDENTICAL) return;
    const double *ga = geo + (size_t)a * GEO_STRIDE, *gb = geo + (size_t)b * GEO_STRIDE;
    const int oa[3] = {P.perm & 3, (P.perm >> 2) & 3, (P.perm >> 4) & 3};
    const int ob[3] = {(P.perm >> 6) & 3, (P.perm >> 8) & 3, (P.perm >> 10) & 3};
    int na_node[3], nb_node[3];
    double A0[3], A1[3], A2[3], B0[3], B1[3], B2[3], na[3], nb[3];
    for (int c = 0; c < 3; ++c) {
        na_node[c] = tris[3 * a + oa[c]];
        nb_node[c] = tris[3 * b + ob[c]];
        A0[c] = ga[3 * oa[0] + c];
        A1[c] = ga[3 * oa[1] + c] - ga[3 * oa[0] + c];
        A2[c] = ga[3 * oa[2] + c] - ga[3 * oa[1] + c];
        B0[c] = gb[3 * ob[0] + c];
        B1[c] = gb[3 * ob[1] + c] - gb[3 * ob[0] + c];
        B2[c] = gb[3 * ob[2] + c] - gb[3 * ob[1] + c];
        na[c] = ga[GEO_N + c];
        nb[c] = gb[GEO_N + c];
    }
    const double scale = 4.0 * ga[GEO_AREA] * gb[GEO_AREA];
    const int npt = tab.n[cls];
    const double *S1 = tab.s1[cls], *S2 = tab.s2[cls], *T1 = tab.t1[cls], *T2 = tab.t2[cls],
                 *W = tab.w[cls];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t EN = (size_t)E * N;

    // weights of point p: (a,b) -> lam_b(t) w rab, (b,a) -> lam_a(s) w rba
    auto point = [&](int p, double &rho, double &irho, double (&wab)[3], double (&wba)[3]) {
        double s1 = S1[p], s2 = S2[p], t1 = T1[p], t2 = T2[p];
        double r[3];
        for (int c = 0; c < 3; ++c)
            r[c] = (A0[c] + s1 * A1[c] + s2 * A2[c]) - (B0[c] + t1 * B1[c] + t2 * B2[c]);
        double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        irho = rsqrt(rr);
        rho = rr * irho;
        double rab = (r[0] * nb[0] + r[1] * nb[1] + r[2] * nb[2]) * irho;
        double rba = -(r[0] * na[0] + r[1] * na[1] + r[2] * na[2]) * irho;
        double w = W[p];
        const double lb[3] = {1.0 - t1, t1 - t2, t2}, la[3] = {1.0 - s1, s1 - s2, s2};
        for (int v = 0; v < 3; ++v) {
            wab[v] = w * rab * lb[v];
            wba[v] = w * rba * la[v];
        }
    };
    auto reduce = [&](double *vals, int nv) {
        for (int k = 0; k < nv; ++k) {
            double v = vals[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < nv) {
            double s = 0.0;
            for (int wi = 0; wi < SS_THREADS / 32; ++wi) s += red[wi][threadIdx.x];
            fin[threadIdx.x] = scale * s;
        }
        __syncthreads();
    };

    // level 0 and the delta = 0 integrand: z[v] (a,b), z[3+v] (b,a), then singular
    double z[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) z[k] = 0.0;
    for (int p = threadIdx.x; p < npt; p += SS_THREADS) {
        double rho, irho, wab[3], wba[3];
        point(p, rho, irho, wab, wba);
        for (int v = 0; v < 3; ++v) {
            z[v] = fma(wab[v], -g.Ap, z[v]);
            z[3 + v] = fma(wba[v], -g.Ap, z[3 + v]);
            z[6 + v] = fma(wab[v], g.Fs * irho * irho, z[6 + v]);
            z[9 + v] = fma(wba[v], g.Fs * irho * irho, z[9 + v]);
        }
    }
    reduce(z, 12);
    double p1[6], p2[6], sing[6];
    for (int k = 0; k < 6; ++k) {
        p1[k] = fin[k];
        p2[k] = 0.0;
        sing[k] = fin[6 + k];
    }
    __syncthreads();

    for (int c0 = 1; c0 <= n_steps; c0 += CH) {
        double acc[6 * CH];
#pragma unroll
        for (int k = 0; k < 6 * CH; ++k) acc[k] = 0.0;
        for (int p = threadIdx.x; p < npt; p += SS_THREADS) {
            double rho, irho, wab[3], wba[3];
            point(p, rho, irho, wab, wba);
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                if (c0 + u <= n_steps) {
                    double v, kf;
                    eval_level(rho, irho, levels + (c0 + u) * LV_STRIDE, g, v, kf);
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        acc[q * CH + u] = fma(wab[q], kf, acc[q * CH + u]);
                        acc[(3 + q) * CH + u] = fma(wba[q], kf, acc[(3 + q) * CH + u]);
                    }
                }
            }
        }
        reduce(acc, 6 * CH);
        if (threadIdx.x == 0) {
            for (int u = 0; u < CH; ++u) {
                int i = c0 + u;
                if (i > n_steps) break;
                for (int k = 0; k < 6; ++k) {
                    double c = fin[k * CH + u];
                    double bk = i == 1 ? g.h * sing[k] - c + p1[k] : 2.0 * p1[k] - c - p2[k];
                    // k < 3: row a, trial node of b; k >= 3: row b, trial node of a
                    const size_t off = (size_t)(i - 1) * EN;
                    if (k < 3)
                        atomic_add_out(K1 + off + (size_t)a * N + nb_node[k], bk);
                    else
                        atomic_add_out(K1 + off + (size_t)b * N + na_node[k - 3], bk);
                    p2[k] = p1[k];
                    p1[k] = c;
                }
            }
        }
        __syncthreads();
    }
}

// --------------------------------------------- hypersingular operator ---
// D_h = D_h^1 + D_h^2 on X_h^{1,0} (Sec. 3.3), blocks [n_steps][N][N].
// D^{1,d} = T^T (alpha^2 V^d (x) I_3) T (eq. D_1_sp_trafo): T holds the
// surface curls of the hat functions, constant on each triangle, so entry
// (i, j) sums alpha^2 (c_{n,i} . c_{m,j}) V^d[n][m] over the triangles n
// around node i and m around node j (node stars, CSR).  One thread per
// (i, j) and chunk of D1_CH blocks: the weight c_{n,i} . c_{m,j} of a star
// pair is formed once and applied to the D1_CH blocks (independent gathers
// from the same row of each block); FP64 sums; the blocks are overwritten.
constexpr int D1_CH = 16;

template <class T>
__global__ void __launch_bounds__(128)
k_hypersingular_d1(const T *__restrict__ V, int E, int N, int n_steps,
                   const int32_t *__restrict__ star_off, const int32_t *__restrict__ star_tri,
                   const double *__restrict__ star_curl, double alpha2, T *__restrict__ D) {
    constexpr int MAX_STAR = 32;
    __shared__ int s_tri[MAX_STAR];
    __shared__ double s_c[MAX_STAR][3];
    const int i = blockIdx.y, d0 = blockIdx.z * D1_CH;
    const int i0 = star_off[i], ni = min(star_off[i + 1] - i0, MAX_STAR);
    for (int t = threadIdx.x; t < ni; t += blockDim.x) {
        s_tri[t] = star_tri[i0 + t];
        for (int o = 0; o < 3; ++o) s_c[t][o] = star_curl[3 * (size_t)(i0 + t) + o];
    }
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const size_t EE = (size_t)E * E;
    const int nd = min(D1_CH, n_steps - d0);
    const T *V0 = V + (size_t)d0 * EE;
    const int j0 = star_off[j], j1 = star_off[j + 1];
    double acc[D1_CH];
#pragma unroll
    for (int u = 0; u < D1_CH; ++u) acc[u] = 0.0;
    for (int b = j0; b < j1; ++b) {
        const int m = star_tri[b];
        const double c0 = star_curl[3 * (size_t)b], c1 = star_curl[3 * (size_t)b + 1],
                     c2 = star_curl[3 * (size_t)b + 2];
        for (int a = 0; a < ni; ++a) {
            const double cc = s_c[a][0] * c0 + s_c[a][1] * c1 + s_c[a][2] * c2;
            const T *p = V0 + (size_t)s_tri[a] * E + m;
            if (nd == D1_CH) {
#pragma unroll
                for (int u = 0; u < D1_CH; ++u) acc[u] = fma(cc, (double)p[u * EE], acc[u]);
            } else {
#pragma unroll
                for (int u = 0; u < D1_CH; ++u)
                    if (u < nd) acc[u] = fma(cc, (double)p[u * EE], acc[u]);
            }
        }
    }
    T *out = D + ((size_t)d0 * N + i) * N + j;
#pragma unroll
    for (int u = 0; u < D1_CH; ++u)
        if (u < nd) out[u * (size_t)N * N] = (T)(alpha2 * acc[u]);
}

// D^{2,d}[i][j] = int int n_x . n_y phi_i(x) phi_j(y) D^{2,d}(x - y) with
// D^{2,0} = alpha (S_0 - S_1), D^{2,d} = alpha (2 S_d - S_{d+1} - S_{d-1}),
// S_i the integral of G^{dtau}(., i h) (eq. D2d with G^{dt} = -G^{dtau}; at
// i = 0 the limit of eq. G_dtau_lim_d, 1/(4 pi alpha rho)), added to D with
// atomics.  Separated pairs: one thread per ordered pair (l, j), the test
// points' barycentric weights summed first per trial point.
__device__ __forceinline__ void atomic_add_d(double *p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_d(float *p, double v) { atomicAdd(p, (float)v); }

template <class OutT>
__global__ void __launch_bounds__(REG_THREADS)
k_regular_d2_f64(const double *__restrict__ geo, const int32_t *__restrict__ tris, int E, int N,
                 const double *__restrict__ rule, int nq, int n_steps, double alpha, double h,
                 OutT *__restrict__ D) {
    __shared__ double xa[4 * MAX_RULE];  // x_a (3) and w_a
    const int l = blockIdx.y;
    const int j = blockIdx.x * REG_THREADS + threadIdx.x;
    const double *gl = geo + (size_t)l * GEO_STRIDE;
    for (int a = threadIdx.x; a < nq; a += REG_THREADS) {
        const double s1 = rule[3 * a], s2 = rule[3 * a + 1];
        for (int c = 0; c < 3; ++c)
            xa[4 * a + c] = gl[GEO_V0 + c] + s1 * (gl[GEO_V1 + c] - gl[GEO_V0 + c]) +
                            s2 * (gl[GEO_V2 + c] - gl[GEO_V1 + c]);
        xa[4 * a + 3] = rule[3 * a + 2];
    }
    __syncthreads();
    if (j >= E) return;
    const int32_t tl[3] = {tris[3 * l], tris[3 * l + 1], tris[3 * l + 2]};
    const int32_t tj[3] = {tris[3 * j], tris[3 * j + 1], tris[3 * j + 2]};
    if (touches(tl, tj)) return;
    const double *gj = geo + (size_t)j * GEO_STRIDE;
    double P0[3], e1[3], e2[3];
    for (int c = 0; c < 3; ++c) {
        P0[c] = gj[GEO_V0 + c];
        e1[c] = gj[GEO_V1 + c] - gj[GEO_V0 + c];
        e2[c] = gj[GEO_V2 + c] - gj[GEO_V1 + c];
    }
    const double nn = gl[GEO_N] * gj[GEO_N] + gl[GEO_N + 1] * gj[GEO_N + 1] + gl[GEO_N + 2] * gj[GEO_N + 2];
    const double c = alpha * nn * 4.0 * gl[GEO_AREA] * gj[GEO_AREA] / (4.0 * 3.14159265358979323846 * alpha);
    const size_t NN = (size_t)N * N;
    double p1[9], p2[9];  // S_{i-1}, S_{i-2}
    for (int i = 0; i <= n_steps; ++i) {
        const double ci = i == 0 ? 0.0 : 0.5 / sqrt(alpha * h * i);  // x = rho ci
        double S[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) S[k] = 0.0;
        for (int b = 0; b < nq; ++b) {
            const double t1 = rule[3 * b], t2 = rule[3 * b + 1], wb = rule[3 * b + 2];
            const double y0 = P0[0] + t1 * e1[0] + t2 * e2[0];
            const double y1 = P0[1] + t1 * e1[1] + t2 * e2[1];
            const double y2 = P0[2] + t1 * e1[2] + t2 * e2[2];
            double sa[3] = {0.0, 0.0, 0.0};
            for (int a = 0; a < nq; ++a) {
                const double r0 = xa[4 * a] - y0, r1 = xa[4 * a + 1] - y1, r2 = xa[4 * a + 2] - y2;
                const double irho = rsqrt(r0 * r0 + r1 * r1 + r2 * r2);
                const double g = xa[4 * a + 3] * irho * (i == 0 ? 1.0 : erf(ci / irho));
                const double s1a = rule[3 * a], s2a = rule[3 * a + 1];
                sa[0] = fma(1.0 - s1a, g, sa[0]);
                sa[1] = fma(s1a - s2a, g, sa[1]);
                sa[2] = fma(s2a, g, sa[2]);
            }
            const double lb[3] = {(1.0 - t1) * wb, (t1 - t2) * wb, t2 * wb};
#pragma unroll
            for (int va = 0; va < 3; ++va)
#pragma unroll
                for (int vb = 0; vb < 3; ++vb) S[3 * va + vb] = fma(sa[va], lb[vb], S[3 * va + vb]);
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) S[k] *= c;
        if (i >= 1) {  // block d = i - 1 is complete
            const int d = i - 1;
#pragma unroll
            for (int va = 0; va < 3; ++va)
#pragma unroll
                for (int vb = 0; vb < 3; ++vb) {
                    const int k = 3 * va + vb;
                    const double v = d == 0 ? p1[k] - S[k] : 2.0 * p1[k] - S[k] - p2[k];
                    atomic_add_d(D + d * NN + (size_t)tl[va] * N + tj[vb], v);
                }
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            p2[k] = p1[k];
            p1[k] = S[k];
        }
    }
}

// Touching pairs: one CTA per unordered pair (a, b) and its regularised rule
// (coordinates s on a, t on b, rotated vertex orders); entry (a, b) and, for
// a != b, the mirrored entry (b, a) receive the same sums.
template <class OutT>
__global__ void __launch_bounds__(SS_THREADS)
k_singular_d2_f64(const double *__restrict__ geo, const int32_t *__restrict__ tris,
                  const TouchPair *__restrict__ pairs, int E, int N, SSTables tab, int n_steps,
                  double alpha, double h, OutT *__restrict__ D) {
    constexpr int CH = 4;
    __shared__ double red[SS_THREADS / 32][9 * CH];
    __shared__ double fin[9 * CH];
    const TouchPair P = pairs[blockIdx.x];
    const int a = P.a, b = P.b, cls = P.cls;
    if (a < 0 || b < a || b >= E || cls < PAIR_VERTEX || cls > PAIR_IDENTICAL) return;
    const double *ga = geo + (size_t)a * GEO_STRIDE, *gb = geo + (size_t)b * GEO_STRIDE;
    const int oa[3] = {P.perm & 3, (P.perm >> 2) & 3, (P.perm >> 4) & 3};
    const int ob[3] = {(P.perm >> 6) & 3, (P.perm >> 8) & 3, (P.perm >> 10) & 3};
    int na_node[3], nb_node[3];
    double A0[3], A1[3], A2[3], B0[3], B1[3], B2[3];
    for (int c = 0; c < 3; ++c) {
        na_node[c] = tris[3 * a + oa[c]];
        nb_node[c] = tris[3 * b + ob[c]];
        A0[c] = ga[3 * oa[0] + c];
        A1[c] = ga[3 * oa[1] + c] - ga[3 * oa[0] + c];
        A2[c] = ga[3 * oa[2] + c] - ga[3 * oa[1] + c];
        B0[c] = gb[3 * ob[0] + c];
        B1[c] = gb[3 * ob[1] + c] - gb[3 * ob[0] + c];
        B2[c] = gb[3 * ob[2] + c] - gb[3 * ob[1] + c];
    }
    const double nn = ga[GEO_N] * gb[GEO_N] + ga[GEO_N + 1] * gb[GEO_N + 1] + ga[GEO_N + 2] * gb[GEO_N + 2];
    const double scale = alpha * nn * 4.0 * ga[GEO_AREA] * gb[GEO_AREA] /
                         (4.0 * 3.14159265358979323846 * alpha);
    const int npt = tab.n[cls];
    const double *S1 = tab.s1[cls], *S2 = tab.s2[cls], *T1 = tab.t1[cls], *T2 = tab.t2[cls],
                 *W = tab.w[cls];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t NN = (size_t)N * N;
    double p1[9], p2[9];
    for (int c0 = 0; c0 <= n_steps; c0 += CH) {
        double acc[9 * CH];
#pragma unroll
        for (int k = 0; k < 9 * CH; ++k) acc[k] = 0.0;
        for (int p = threadIdx.x; p < npt; p += SS_THREADS) {
            const double s1 = S1[p], s2 = S2[p], t1 = T1[p], t2 = T2[p];
            double r[3];
            for (int c = 0; c < 3; ++c)
                r[c] = (A0[c] + s1 * A1[c] + s2 * A2[c]) - (B0[c] + t1 * B1[c] + t2 * B2[c]);
            const double irho = rsqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            const double la[3] = {1.0 - s1, s1 - s2, s2}, lb[3] = {1.0 - t1, t1 - t2, t2};
            const double w = W[p] * irho;
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int i = c0 + u;
                if (i > n_steps) break;
                const double g = w * (i == 0 ? 1.0 : erf(0.5 / (irho * sqrt(alpha * h * i))));
#pragma unroll
                for (int va = 0; va < 3; ++va)
#pragma unroll
                    for (int vb = 0; vb < 3; ++vb)
                        acc[9 * u + 3 * va + vb] = fma(la[va] * lb[vb], g, acc[9 * u + 3 * va + vb]);
            }
        }
        for (int k = 0; k < 9 * CH; ++k) {
            double v = acc[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < 9 * CH) {
            double sum = 0.0;
            for (int wi = 0; wi < SS_THREADS / 32; ++wi) sum += red[wi][threadIdx.x];
            fin[threadIdx.x] = scale * sum;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int u = 0; u < CH; ++u) {
                const int i = c0 + u;
                if (i > n_steps) break;
                for (int k = 0; k < 9; ++k) {
                    const double S = fin[9 * u + k];
                    if (i >= 1) {
                        const int d = i - 1;
                        const double v = d == 0 ? p1[k] - S : 2.0 * p1[k] - S - p2[k];
                        const int va = k / 3, vb = k % 3;
                        atomic_add_d(D + d * NN + (size_t)na_node[va] * N + nb_node[vb], v);
                        if (cls != PAIR_IDENTICAL)
                            atomic_add_d(D + d * NN + (size_t)nb_node[vb] * N + na_node[va], v);
                    }
                    p2[k] = p1[k];
                    p1[k] = S;
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------ non-uniform time grids ---
// On a grid t_0 = 0 < t_1 < ... < t_n the blocks A^{k,i} (k >= i, packed at
// b(k,i) = k(k+1)/2 + i) are four-corner combinations of the spatial sums S
// of G^{dtau dt} (and of its scaled normal derivative) at the time
// differences t_a - t_b; the diagonal adds h_k times the delta = 0
// singular sums (eq. V0 / eq. K0 with the local step).  The host lists the
// distinct differences ("levels", level 0 = delta 0) and, per level, the
// blocks it enters with its coefficient (CSR); a thread that owns the entry
// (l, j) of every block evaluates each level once and adds it to the blocks
// of its list.  The blocks must start at zero; FP64 storage only (the
// corner terms cancel).
struct NuLists {
    const double *levels;      // [n_levels][LV_STRIDE]
    const int32_t *off;        // [n_levels + 2]: levels 0..n_levels-1, then the singular list
    const int32_t *blk;
    const double *coef;
    int n_levels;
};

template <int CH>
__global__ void __launch_bounds__(REG_THREADS)
k_regular_nu_f64(const double *__restrict__ geo, const int32_t *__restrict__ tris, int E,
                 const double *__restrict__ rule, int nq, NuLists lists, Globals g,
                 double *__restrict__ V, double *__restrict__ K) {
    __shared__ double xa[4 * MAX_RULE];
    const int l = blockIdx.y;
    const int j = blockIdx.x * REG_THREADS + threadIdx.x;
    const double *gl = geo + (size_t)l * GEO_STRIDE;
    for (int a = threadIdx.x; a < nq; a += REG_THREADS) {
        double s1 = rule[3 * a], s2 = rule[3 * a + 1];
        for (int c = 0; c < 3; ++c)
            xa[4 * a + c] = gl[GEO_V0 + c] + s1 * (gl[GEO_V1 + c] - gl[GEO_V0 + c]) +
                            s2 * (gl[GEO_V2 + c] - gl[GEO_V1 + c]);
        xa[4 * a + 3] = rule[3 * a + 2];
    }
    __syncthreads();
    if (j >= E) return;
    const int32_t tl[3] = {tris[3 * l], tris[3 * l + 1], tris[3 * l + 2]};
    const int32_t tj[3] = {tris[3 * j], tris[3 * j + 1], tris[3 * j + 2]};
    if (touches(tl, tj)) return;
    const double *gj = geo + (size_t)j * GEO_STRIDE;
    double P0[3], e1[3], e2[3], n[3];
    for (int c = 0; c < 3; ++c) {
        P0[c] = gj[GEO_V0 + c];
        e1[c] = gj[GEO_V1 + c] - gj[GEO_V0 + c];
        e2[c] = gj[GEO_V2 + c] - gj[GEO_V1 + c];
        n[c] = gj[GEO_N + c];
    }
    const double scale = 4.0 * gl[GEO_AREA] * gj[GEO_AREA];
    const size_t EE = (size_t)E * E, ij = (size_t)l * E + j;
    auto add = [&](int L, double sv, double sk) {
        for (int e = lists.off[L]; e < lists.off[L + 1]; ++e) {
            const size_t o = (size_t)lists.blk[e] * EE + ij;
            V[o] += lists.coef[e] * sv;
            K[o] += lists.coef[e] * sk;
        }
    };
    // level 0 (delta -> 0 limits) and the delta = 0 singular sums
    double s0v = 0, s0k = 0, ssv = 0, ssk = 0;
    for (int b = 0; b < nq; ++b) {
        double t1 = rule[3 * b], t2 = rule[3 * b + 1], wb = rule[3 * b + 2];
        double y0 = P0[0] + t1 * e1[0] + t2 * e2[0];
        double y1 = P0[1] + t1 * e1[1] + t2 * e2[1];
        double y2 = P0[2] + t1 * e1[2] + t2 * e2[2];
        for (int a = 0; a < nq; ++a) {
            double r0 = xa[4 * a] - y0, r1 = xa[4 * a + 1] - y1, r2 = xa[4 * a + 2] - y2;
            double rr = r0 * r0 + r1 * r1 + r2 * r2;
            double irho = rsqrt(rr), rho = rr * irho;
            double rnr = (r0 * n[0] + r1 * n[1] + r2 * n[2]) * irho;
            double w = xa[4 * a + 3] * wb;
            s0v = fma(w, g.A * rho, s0v);
            s0k = fma(w, -g.Ap * rnr, s0k);
            ssv = fma(w, g.F * irho, ssv);
            ssk = fma(w, g.Fs * rnr * irho * irho, ssk);
        }
    }
    add(0, scale * s0v, scale * s0k);
    add(lists.n_levels, scale * ssv, scale * ssk);
    for (int c0 = 1; c0 < lists.n_levels; c0 += CH) {
        double sv[CH], sk[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) sv[u] = sk[u] = 0.0;
        for (int b = 0; b < nq; ++b) {
            double t1 = rule[3 * b], t2 = rule[3 * b + 1], wb = rule[3 * b + 2];
            double y0 = P0[0] + t1 * e1[0] + t2 * e2[0];
            double y1 = P0[1] + t1 * e1[1] + t2 * e2[1];
            double y2 = P0[2] + t1 * e1[2] + t2 * e2[2];
            for (int a = 0; a < nq; ++a) {
                double r0 = xa[4 * a] - y0, r1 = xa[4 * a + 1] - y1, r2 = xa[4 * a + 2] - y2;
                double rr = r0 * r0 + r1 * r1 + r2 * r2;
                double irho = rsqrt(rr), rho = rr * irho;
                double rnr = (r0 * n[0] + r1 * n[1] + r2 * n[2]) * irho;
                double w = xa[4 * a + 3] * wb, wk = w * rnr;
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    if (c0 + u < lists.n_levels) {
                        double v, kf;
                        eval_level(rho, irho, lists.levels + (c0 + u) * LV_STRIDE, g, v, kf);
                        sv[u] = fma(w, v, sv[u]);
                        sk[u] = fma(wk, kf, sk[u]);
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < CH; ++u)
            if (c0 + u < lists.n_levels) add(c0 + u, scale * sv[u], scale * sk[u]);
    }
}

template <int CH>
__global__ void __launch_bounds__(SS_THREADS)
k_singular_nu_f64(const double *__restrict__ geo, const TouchPair *__restrict__ pairs, int E,
                  SSTables tab, NuLists lists, Globals g, double *__restrict__ V,
                  double *__restrict__ K) {
    __shared__ double red[SS_THREADS / 32][3 * CH + 8];
    __shared__ double fin[3 * CH + 8];
    const TouchPair P = pairs[blockIdx.x];
    const int a = P.a, b = P.b, cls = P.cls;
    if (a < 0 || b < a || b >= E || cls < PAIR_VERTEX || cls > PAIR_IDENTICAL) return;
    const double *ga = geo + (size_t)a * GEO_STRIDE, *gb = geo + (size_t)b * GEO_STRIDE;
    double A0[3], A1[3], A2[3], B0[3], B1[3], B2[3], na[3], nb[3];
    {
        int oa0 = P.perm & 3, oa1 = (P.perm >> 2) & 3, oa2 = (P.perm >> 4) & 3;
        int ob0 = (P.perm >> 6) & 3, ob1 = (P.perm >> 8) & 3, ob2 = (P.perm >> 10) & 3;
        for (int c = 0; c < 3; ++c) {
            A0[c] = ga[3 * oa0 + c];
            A1[c] = ga[3 * oa1 + c] - ga[3 * oa0 + c];
            A2[c] = ga[3 * oa2 + c] - ga[3 * oa1 + c];
            B0[c] = gb[3 * ob0 + c];
            B1[c] = gb[3 * ob1 + c] - gb[3 * ob0 + c];
            B2[c] = gb[3 * ob2 + c] - gb[3 * ob1 + c];
            na[c] = ga[GEO_N + c];
            nb[c] = gb[GEO_N + c];
        }
    }
    const double scale = 4.0 * ga[GEO_AREA] * gb[GEO_AREA];
    const bool ident = cls == PAIR_IDENTICAL;
    const int npt = tab.n[cls];
    const double *S1 = tab.s1[cls], *S2 = tab.s2[cls], *T1 = tab.t1[cls], *T2 = tab.t2[cls],
                 *W = tab.w[cls];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t EE = (size_t)E * E, iab = (size_t)a * E + b, iba = (size_t)b * E + a;
    auto point = [&](int p, double &rho, double &irho, double &rab, double &rba, double &w) {
        double s1 = S1[p], s2 = S2[p], t1 = T1[p], t2 = T2[p];
        double r[3];
        for (int c = 0; c < 3; ++c)
            r[c] = (A0[c] + s1 * A1[c] + s2 * A2[c]) - (B0[c] + t1 * B1[c] + t2 * B2[c]);
        double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        irho = rsqrt(rr);
        rho = rr * irho;
        rab = (r[0] * nb[0] + r[1] * nb[1] + r[2] * nb[2]) * irho;
        rba = -(r[0] * na[0] + r[1] * na[1] + r[2] * na[2]) * irho;
        w = W[p];
    };
    auto reduce = [&](double *vals, int nv) {
        for (int k = 0; k < nv; ++k) {
            double v = vals[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < nv) {
            double s = 0.0;
            for (int wi = 0; wi < SS_THREADS / 32; ++wi) s += red[wi][threadIdx.x];
            fin[threadIdx.x] = scale * s;
        }
        __syncthreads();
    };
    // thread 0 adds level L's sums (V, K at (a,b), K at (b,a)) to its blocks
    auto add = [&](int L, double cv, double ca, double cb) {
        for (int e = lists.off[L]; e < lists.off[L + 1]; ++e) {
            const size_t o = (size_t)lists.blk[e] * EE;
            const double c = lists.coef[e];
            V[o + iab] += c * cv;
            if (!ident) {
                V[o + iba] += c * cv;
                K[o + iab] += c * ca;
                K[o + iba] += c * cb;
            }
        }
    };
    double z[6] = {0, 0, 0, 0, 0, 0};
    for (int p = threadIdx.x; p < npt; p += SS_THREADS) {
        double rho, irho, rab, rba, w;
        point(p, rho, irho, rab, rba, w);
        z[0] = fma(w, g.A * rho, z[0]);
        z[1] = fma(w, -g.Ap * rab, z[1]);
        z[2] = fma(w, -g.Ap * rba, z[2]);
        z[3] = fma(w, g.F * irho, z[3]);
        z[4] = fma(w, g.Fs * rab * irho * irho, z[4]);
        z[5] = fma(w, g.Fs * rba * irho * irho, z[5]);
    }
    reduce(z, 6);
    if (threadIdx.x == 0) {
        add(0, fin[0], fin[1], fin[2]);
        add(lists.n_levels, fin[3], fin[4], fin[5]);
    }
    __syncthreads();
    for (int c0 = 1; c0 < lists.n_levels; c0 += CH) {
        double acc[3 * CH];
#pragma unroll
        for (int k = 0; k < 3 * CH; ++k) acc[k] = 0.0;
        for (int p = threadIdx.x; p < npt; p += SS_THREADS) {
            double rho, irho, rab, rba, w;
            point(p, rho, irho, rab, rba, w);
            double wa = w * rab, wb = w * rba;
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                if (c0 + u < lists.n_levels) {
                    double v, kf;
                    eval_level(rho, irho, lists.levels + (c0 + u) * LV_STRIDE, g, v, kf);
                    acc[u] = fma(w, v, acc[u]);
                    acc[CH + u] = fma(wa, kf, acc[CH + u]);
                    acc[2 * CH + u] = fma(wb, kf, acc[2 * CH + u]);
                }
            }
        }
        reduce(acc, 3 * CH);
        if (threadIdx.x == 0)
            for (int u = 0; u < CH && c0 + u < lists.n_levels; ++u)
                add(c0 + u, fin[u], fin[CH + u], fin[2 * CH + u]);
        __syncthreads();
    }
}

template <class OutT>
static stb_status run_assembly(const Mesh &m, const stb_params &p, OutT *V, OutT *K,
                               const AssemblyLayout &L, int32_t *status, cudaStream_t s) {
    constexpr int CH = 8;
    const int E = (int)m.n_tris;
    const int nq = p.quad_regular * p.quad_regular;
    Globals g = make_globals(p);
    size_t smem = sizeof(double) * (4 * MAX_RULE + (size_t)(p.n_steps + 1) * LV_STRIDE);
    STB_CUDA(cudaFuncSetAttribute(k_regular_f64<CH, OutT>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((E + REG_THREADS - 1) / REG_THREADS, E);
    count_launch(s);
    k_regular_f64<CH, OutT><<<grid, REG_THREADS, smem, s>>>(L.geo, m.d_tris, E, L.rule, nq,
                                                            L.levels, p.n_steps, g, V, K);
    stb_status st = check_launch("k_regular_f64");
    if (st) return st;
    if (m.n_touch > 0) {
        SSTables tab{};
        const double *base = L.ss;
        for (int cls = 1; cls <= 3; ++cls) {
            size_t n = L.ss_n[cls];
            tab.s1[cls] = base;
            tab.s2[cls] = base + n;
            tab.t1[cls] = base + 2 * n;
            tab.t2[cls] = base + 3 * n;
            tab.w[cls] = base + 4 * n;
            tab.n[cls] = (int)n;
            base += 5 * n;
        }
        count_launch(s);
        k_singular_f64<CH, OutT><<<(unsigned)m.n_touch, SS_THREADS, 0, s>>>(
            L.geo, L.pairs, E, tab, L.levels, p.n_steps, g, V, K);
        if ((st = check_launch("k_singular_f64"))) return st;
    }
    return STB_OK;
}

template <class OutT>
static stb_status run_assembly_k1(const Mesh &m, const stb_params &p, OutT *K1,
                                  const AssemblyLayout &L, cudaStream_t s) {
    constexpr int CH = 8;
    const int E = (int)m.n_tris, N = (int)m.n_nodes;
    const int nq = p.quad_regular * p.quad_regular;
    Globals g = make_globals(p);
    STB_CUDA(cudaMemsetAsync(K1, 0, sizeof(OutT) * (size_t)p.n_steps * E * N, s));
    size_t smem = sizeof(double) * (4 * MAX_RULE + (size_t)(p.n_steps + 1) * LV_STRIDE);
    STB_CUDA(cudaFuncSetAttribute(k_regular_k1_f64<CH, OutT>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((E + REG_THREADS - 1) / REG_THREADS, E);
    count_launch(s);
    k_regular_k1_f64<CH, OutT><<<grid, REG_THREADS, smem, s>>>(L.geo, m.d_tris, E, N, L.rule, nq,
                                                               L.levels, p.n_steps, g, K1);
    stb_status st = check_launch("k_regular_k1_f64");
    if (st || m.n_touch == 0) return st;
    SSTables tab{};
    const double *base = L.ss;
    for (int cls = 1; cls <= 3; ++cls) {
        size_t n = L.ss_n[cls];
        tab.s1[cls] = base;
        tab.s2[cls] = base + n;
        tab.t1[cls] = base + 2 * n;
        tab.t2[cls] = base + 3 * n;
        tab.w[cls] = base + 4 * n;
        tab.n[cls] = (int)n;
        base += 5 * n;
    }
    count_launch(s);
    k_singular_k1_f64<CH, OutT><<<(unsigned)m.n_touch, SS_THREADS, 0, s>>>(
        L.geo, m.d_tris, L.pairs, E, N, tab, L.levels, p.n_steps, g, K1);
    return check_launch("k_singular_k1_f64");
}

// Node stars of the mesh for D^1: for node i the triangles around it
// (CSR) and the surface curl of phi_i on each, curl phi_v = (P_{v+1} -
// P_{v+2}) / (2 Delta) (the in-plane gradient of the barycentric
// coordinate turned by the normal; vertices cyclic, counter-clockwise).
struct NodeStars {
    std::vector<int32_t> off, tri;
    std::vector<double> curl;
    int max_star = 0;
};

static NodeStars node_stars(const Mesh &m) {
    NodeStars S;
    const int64_t N = m.n_nodes, E = m.n_tris;
    S.off.assign(N + 1, 0);
    for (int64_t e = 0; e < E; ++e)
        for (int v = 0; v < 3; ++v) ++S.off[m.tris[3 * e + v] + 1];
    for (int64_t i = 0; i < N; ++i) {
        S.max_star = std::max(S.max_star, S.off[i + 1]);
        S.off[i + 1] += S.off[i];
    }
    S.tri.assign(3 * E, 0);
    S.curl.assign(9 * E, 0.0);
    std::vector<int32_t> fill(S.off.begin(), S.off.end() - 1);
    for (int64_t e = 0; e < E; ++e) {
        const double *P[3];
        for (int v = 0; v < 3; ++v) P[v] = m.nodes.data() + 3 * (size_t)m.tris[3 * e + v];
        const double u[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
        const double w[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
        const double cx = u[1] * w[2] - u[2] * w[1], cy = u[2] * w[0] - u[0] * w[2],
                     cz = u[0] * w[1] - u[1] * w[0];
        const double two_area = std::sqrt(cx * cx + cy * cy + cz * cz);
        for (int v = 0; v < 3; ++v) {
            const int32_t i = m.tris[3 * e + v];
            const int32_t b = fill[i]++;
            S.tri[b] = (int32_t)e;
            const double *A = P[(v + 1) % 3], *B = P[(v + 2) % 3];
            for (int o = 0; o < 3; ++o) S.curl[3 * (size_t)b + o] = (A[o] - B[o]) / two_area;
        }
    }
    return S;
}

template <class OutT>
static stb_status run_hypersingular(const Mesh &m, const stb_params &p, const OutT *V, OutT *D,
                                    const AssemblyLayout &L, const AssemblyLayout *Lmix,
                                    const float *coords, const int32_t *star_off,
                                    const int32_t *star_tri, const double *star_curl,
                                    cudaStream_t s) {
    const int E = (int)m.n_tris, N = (int)m.n_nodes;
    const double h = p.T / p.n_steps;
    dim3 g1((N + 127) / 128, N, (p.n_steps + D1_CH - 1) / D1_CH);
    count_launch(s);
    k_hypersingular_d1<OutT><<<g1, 128, 0, s>>>(V, E, N, p.n_steps, star_off, star_tri,
                                               star_curl, p.alpha * p.alpha, D);
    stb_status st = check_launch("k_hypersingular_d1");
    if (st) return st;
    if constexpr (std::is_same<OutT, float>::value) {
        if (Lmix) {  // mixed precision: separated and touching pairs
            stb_params pm = p;
            pm.precision = STB_PREC_MIXED;
            if ((st = run_d2_regular_mixed(m, pm, D, *Lmix, s))) return st;
            return run_d2_singular_mixed(m, pm, D, *Lmix, coords, s);
        }
    }
    if (!Lmix) {
        dim3 g2((E + REG_THREADS - 1) / REG_THREADS, E);
        count_launch(s);
        k_regular_d2_f64<OutT><<<g2, REG_THREADS, 0, s>>>(L.geo, m.d_tris, E, N, L.rule,
                                                           p.quad_regular * p.quad_regular,
                                                           p.n_steps, p.alpha, h, D);
        if ((st = check_launch("k_regular_d2_f64"))) return st;
    }
    if (m.n_touch == 0) return STB_OK;
    SSTables tab{};
    const double *base = L.ss;
    for (int cls = 1; cls <= 3; ++cls) {
        size_t n = L.ss_n[cls];
        tab.s1[cls] = base;
        tab.s2[cls] = base + n;
        tab.t1[cls] = base + 2 * n;
        tab.t2[cls] = base + 3 * n;
        tab.w[cls] = base + 4 * n;
        tab.n[cls] = (int)n;
        base += 5 * n;
    }
    count_launch(s);
    k_singular_d2_f64<OutT><<<(unsigned)m.n_touch, SS_THREADS, 0, s>>>(
        L.geo, m.d_tris, L.pairs, E, N, tab, p.n_steps, p.alpha, h, D);
    return check_launch("k_singular_d2_f64");
}

}  // namespace stb

using namespace stb;

// FP64 path: upload the host tables (regular rule, regularised rules, level
// constants), then geometry and pair classification.
stb_status stb::prepare_fp64(const Mesh &m, const stb_params &p, const AssemblyLayout &L,
                             int32_t *status, cudaStream_t s) {
    upload_psi_coeffs(s);
    stb_status st;
    // FP64 host tables: regular rule, regularised rules, level constants
    std::vector<double> host;
    {
        std::vector<double> a, b, c, d, w;
        triangle_rule(p.quad_regular, a, b, w);
        for (size_t i = 0; i < w.size(); ++i) {
            host.push_back(a[i]);
            host.push_back(b[i]);
            host.push_back(w[i]);
        }
        size_t rule_pad = (size_t)((char *)L.ss - (char *)L.rule) / sizeof(double);
        host.resize(rule_pad, 0.0);
        for (int cls = 1; cls <= 3; ++cls) {
            ss_rule(cls, p.quad_singular, a, b, c, d, w);
            host.insert(host.end(), a.begin(), a.end());
            host.insert(host.end(), b.begin(), b.end());
            host.insert(host.end(), c.begin(), c.end());
            host.insert(host.end(), d.begin(), d.end());
            host.insert(host.end(), w.begin(), w.end());
        }
        size_t lev_pad = (size_t)((char *)L.levels - (char *)L.rule) / sizeof(double);
        host.resize(lev_pad, 0.0);
        const double pi = 3.14159265358979323846, al = p.alpha;
        const double h = p.T / p.n_steps;
        for (int i = 0; i <= p.n_steps; ++i) {
            double lvv[LV_STRIDE] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (i > 0) {
                double delta = i * h, sd = std::sqrt(delta);
                lvv[LV_C] = 1.0 / (2.0 * std::sqrt(al * delta));
                lvv[LV_B] = delta / (4.0 * pi * al);
                lvv[LV_CC] = sd / (4.0 * pi * std::sqrt(pi * al * al * al));
                lvv[LV_D] = delta / (4.0 * pi);
                lvv[LV_E] = sd / (4.0 * pi * std::sqrt(pi * al));
            }
            host.insert(host.end(), lvv, lvv + LV_STRIDE);
        }
    }
    STB_CUDA(cudaMemcpyAsync(L.rule, host.data(), host.size() * sizeof(double),
                             cudaMemcpyHostToDevice, s));
    STB_CUDA(cudaMemsetAsync(L.pairs, 0xff, sizeof(TouchPair) * (m.n_touch > 0 ? m.n_touch : 1), s));
    if ((st = launch_geometry(m, L.geo, s))) return st;
    if ((st = launch_classify(m, L.row_count, L.row_off, L.pairs, status, s))) return st;
    return STB_OK;
}

// Mixed path: upload the FP32 tables, then geometry and pair classification.
stb_status stb::prepare_mixed(const Mesh &m, const stb_params &p, const AssemblyLayout &L,
                         int32_t *status, cudaStream_t s) {
    upload_psi_coeffs(s);
    std::vector<float> rule, ss, nodes, host;
    mixed_tables(p, rule, ss, nodes);
    host = rule;
    host.resize((size_t)(L.mss - L.mrule), 0.f);
    host.insert(host.end(), ss.begin(), ss.end());
    host.resize((size_t)(L.mnodes - L.mrule), 0.f);
    host.insert(host.end(), nodes.begin(), nodes.end());
    STB_CUDA(cudaMemcpyAsync(L.mrule, host.data(), host.size() * sizeof(float),
                             cudaMemcpyHostToDevice, s));
    STB_CUDA(cudaMemsetAsync(L.pairs, 0xff, sizeof(TouchPair) * (m.n_touch > 0 ? m.n_touch : 1), s));
    stb_status st = launch_geometry(m, L.geo, s);
    if (st) return st;
    return launch_classify(m, L.row_count, L.row_off, L.pairs, status, s);
}

extern "C" stb_status stb_assemble_workspace_size(const stb_mesh *mesh, const stb_params *params,
                                                  size_t *bytes) {
    if (!mesh || !bytes) return fail(STB_ERR_INVALID_ARG, "mesh and bytes must be given");
    stb_status st = check_assembly_params(params);
    if (st) return st;
    *bytes = align256(assembly_layout(mesh->m, *params, nullptr, 0).bytes);
    return STB_OK;
}

extern "C" stb_status stb_assemble(const stb_mesh *mesh, const stb_params *params, void *V, void *K,
                                   void *ws, size_t ws_bytes, stb_stream stream) {
    if (!mesh || !V) return fail(STB_ERR_INVALID_ARG, "mesh and V must be given");
    stb_status st = check_assembly_params(params);
    if (st) return st;
    const Mesh &m = mesh->m;
    if (m.n_tris > 65535) return fail(STB_ERR_INVALID_ARG, "dense assembly supports E <= 65535");
    AssemblyLayout L = assembly_layout(m, *params, ws, ws_bytes);
    if ((st = check_workspace(ws, ws_bytes, L.bytes))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    upload_psi_coeffs(s);

    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    int32_t *status = status_word(ws);
    if (params->precision == STB_PREC_MIXED) {
        if ((st = prepare_mixed(m, *params, L, status, s))) return st;
        return run_assembly_mixed(m, *params, V, K, L, s);
    }
    if ((st = prepare_fp64(m, *params, L, status, s))) return st;
    if (params->storage == STB_STORE_F64)
        return run_assembly<double>(m, *params, (double *)V, (double *)K, L, status, s);
    return run_assembly<float>(m, *params, (float *)V, (float *)K, L, status, s);
}

// Coordinates of the regularised rules for the mixed piecewise-linear K:
// (s1, s2, t1, t2) per class 1..3.
static size_t k1_coords_floats(const stb_params &p) {
    size_t n = 0;
    for (int cls = 1; cls <= 3; ++cls) n += 4 * (size_t)ss_rule_size(cls, p.quad_singular);
    return n;
}

extern "C" stb_status stb_assemble_k1_workspace_size(const stb_mesh *mesh, const stb_params *params,
                                                     size_t *bytes) {
    if (!mesh || !bytes || !params) return fail(STB_ERR_INVALID_ARG, "mesh, params and bytes must be given");
    stb_status st = check_assembly_params(params);
    if (st) return st;
    if (params->precision == STB_PREC_MIXED && params->storage != STB_STORE_F32)
        return fail(STB_ERR_INVALID_ARG, "mixed precision needs STB_STORE_F32 blocks");
    *bytes = align256(assembly_layout(mesh->m, *params, nullptr, 0).bytes) +
             (params->precision == STB_PREC_MIXED ? align256(k1_coords_floats(*params) * 4) : 0);
    return STB_OK;
}

extern "C" stb_status stb_assemble_k1(const stb_mesh *mesh, const stb_params *params, void *K1,
                                      void *ws, size_t ws_bytes, stb_stream stream) {
    if (!mesh || !K1) return fail(STB_ERR_INVALID_ARG, "mesh and K1 must be given");
    size_t need;
    stb_status st = stb_assemble_k1_workspace_size(mesh, params, &need);
    if (st) return st;
    if ((st = check_workspace(ws, ws_bytes, need))) return st;
    const Mesh &m = mesh->m;
    if (m.n_tris > 65535) return fail(STB_ERR_INVALID_ARG, "dense assembly supports E <= 65535");
    AssemblyLayout L = assembly_layout(m, *params, ws, ws_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    if (params->precision == STB_PREC_MIXED) {
        if ((st = prepare_mixed(m, *params, L, status_word(ws), s))) return st;
        // the rules' coordinates, FP32, behind the assembly layout
        float *coords = reinterpret_cast<float *>(static_cast<char *>(ws) + align256(L.bytes));
        std::vector<float> host;
        std::vector<double> s1, s2, t1, t2, w;
        for (int cls = 1; cls <= 3; ++cls) {
            ss_rule(cls, params->quad_singular, s1, s2, t1, t2, w);
            for (auto *v : {&s1, &s2, &t1, &t2})
                for (double x : *v) host.push_back((float)x);
        }
        STB_CUDA(cudaMemcpyAsync(coords, host.data(), host.size() * sizeof(float),
                                 cudaMemcpyHostToDevice, s));
        return run_assembly_k1_mixed(m, *params, (float *)K1, L, coords, s);
    }
    if ((st = prepare_fp64(m, *params, L, status_word(ws), s))) return st;
    if (params->storage == STB_STORE_F64) return run_assembly_k1<double>(m, *params, (double *)K1, L, s);
    return run_assembly_k1<float>(m, *params, (float *)K1, L, s);
}

// ---- hypersingular operator (Sec. 3.3) --------------------------------------
static size_t stars_bytes(const Mesh &m) {
    return align256(sizeof(int32_t) * (m.n_nodes + 1)) + align256(sizeof(int32_t) * 3 * m.n_tris) +
           align256(sizeof(double) * 9 * m.n_tris);
}

extern "C" stb_status stb_assemble_d_workspace_size(const stb_mesh *mesh, const stb_params *params,
                                                    size_t *bytes) {
    if (!mesh || !bytes || !params) return fail(STB_ERR_INVALID_ARG, "mesh, params and bytes must be given");
    stb_status st = check_assembly_params(params);
    if (st) return st;
    if (params->precision == STB_PREC_MIXED && params->storage != STB_STORE_F32)
        return fail(STB_ERR_INVALID_ARG, "mixed precision needs STB_STORE_F32 blocks");
    if (mesh->m.n_nodes > 65535) return fail(STB_ERR_INVALID_ARG, "n_nodes must be <= 65535");
    stb_params p64 = *params;
    p64.precision = STB_PREC_FP64;
    *bytes = align256(assembly_layout(mesh->m, p64, nullptr, 0).bytes) + stars_bytes(mesh->m);
    if (params->precision == STB_PREC_MIXED)
        *bytes += align256(assembly_layout(mesh->m, *params, nullptr, 0).bytes) +
                  align256(k1_coords_floats(*params) * 4);
    return STB_OK;
}

extern "C" stb_status stb_assemble_d(const stb_mesh *mesh, const stb_params *params, const void *V,
                                     void *D, void *ws, size_t ws_bytes, stb_stream stream) {
    if (!mesh || !V || !D) return fail(STB_ERR_INVALID_ARG, "mesh, V and D must be given");
    size_t need;
    stb_status st = stb_assemble_d_workspace_size(mesh, params, &need);
    if (st) return st;
    if ((st = check_workspace(ws, ws_bytes, need))) return st;
    const Mesh &m = mesh->m;
    if (m.n_tris > 65535) return fail(STB_ERR_INVALID_ARG, "dense assembly supports E <= 65535");
    const NodeStars S = node_stars(m);
    if (S.max_star > 32) return fail(STB_ERR_INVALID_ARG, "a node belongs to more than 32 triangles");
    // FP64 tables (touching pairs, and separated pairs in FP64), then the
    // node stars, then (mixed) a second problem layout with the FP32 tables
    stb_params p64 = *params;
    p64.precision = STB_PREC_FP64;
    AssemblyLayout L = assembly_layout(m, p64, ws, ws_bytes);
    char *p = static_cast<char *>(ws) + align256(L.bytes);
    int32_t *star_off = reinterpret_cast<int32_t *>(p);
    p += align256(sizeof(int32_t) * (m.n_nodes + 1));
    int32_t *star_tri = reinterpret_cast<int32_t *>(p);
    p += align256(sizeof(int32_t) * 3 * m.n_tris);
    double *star_curl = reinterpret_cast<double *>(p);
    p += align256(sizeof(double) * 9 * m.n_tris);
    const bool mixed = params->precision == STB_PREC_MIXED;
    AssemblyLayout Lm{};
    float *coords = nullptr;
    if (mixed) {  // Carve starts 256 bytes in: the status word of this sub-layout is unused
        const size_t off = (size_t)(p - static_cast<char *>(ws));
        Lm = assembly_layout(m, *params, p, ws_bytes - off);
        coords = reinterpret_cast<float *>(p + align256(Lm.bytes));
    }
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    if ((st = prepare_fp64(m, p64, L, status_word(ws), s))) return st;
    if (mixed) {
        if ((st = prepare_mixed(m, *params, Lm, status_word(ws), s))) return st;
        std::vector<float> host;
        std::vector<double> s1, s2, t1, t2, w;
        for (int cls = 1; cls <= 3; ++cls) {
            ss_rule(cls, params->quad_singular, s1, s2, t1, t2, w);
            for (auto *v : {&s1, &s2, &t1, &t2})
                for (double x : *v) host.push_back((float)x);
        }
        STB_CUDA(cudaMemcpyAsync(coords, host.data(), host.size() * sizeof(float),
                                 cudaMemcpyHostToDevice, s));
    }
    STB_CUDA(cudaMemcpyAsync(star_off, S.off.data(), sizeof(int32_t) * S.off.size(),
                             cudaMemcpyHostToDevice, s));
    STB_CUDA(cudaMemcpyAsync(star_tri, S.tri.data(), sizeof(int32_t) * S.tri.size(),
                             cudaMemcpyHostToDevice, s));
    STB_CUDA(cudaMemcpyAsync(star_curl, S.curl.data(), sizeof(double) * S.curl.size(),
                             cudaMemcpyHostToDevice, s));
    if (params->storage == STB_STORE_F64)
        st = run_hypersingular<double>(m, p64, (const double *)V, (double *)D, L, nullptr,
                                       nullptr, star_off, star_tri, star_curl, s);
    else
        st = run_hypersingular<float>(m, p64, (const float *)V, (float *)D, L,
                                      mixed ? &Lm : nullptr, coords, star_off, star_tri,
                                      star_curl, s);
    if (st) return st;
    // the host tables above are copied from pageable memory before the
    // copies return; nothing else refers to them
    return STB_OK;
}

// ---- V and the right-hand side without K (matrix-free K g) -------------------
extern "C" stb_status stb_assemble_vrhs_workspace_size(const stb_mesh *mesh,
                                                       const stb_params *params, int32_t nrhs,
                                                       size_t *bytes) {
    if (!mesh || !bytes || !params) return fail(STB_ERR_INVALID_ARG, "mesh, params and bytes must be given");
    stb_status st = check_assembly_params(params);
    if (st) return st;
    if (params->precision != STB_PREC_MIXED || params->storage != STB_STORE_F32)
        return fail(STB_ERR_INVALID_ARG, "the matrix-free right-hand side needs STB_PREC_MIXED and STB_STORE_F32");
    if (nrhs < 1 || (int64_t)nrhs * params->n_steps > 128)
        return fail(STB_ERR_INVALID_ARG, "need 1 <= nrhs and nrhs * n_steps <= 128");
    if (params->quad_regular * params->quad_regular > 256)
        return fail(STB_ERR_INVALID_ARG, "quad_regular must be <= 16");
    *bytes = align256(assembly_layout(mesh->m, *params, nullptr, 0).bytes);
    return STB_OK;
}

extern "C" stb_status stb_assemble_vrhs(const stb_mesh *mesh, const stb_params *params, void *V,
                                        const double *g, int32_t nrhs, double *f, void *ws,
                                        size_t ws_bytes, stb_stream stream) {
    if (!mesh || !V || !g || !f) return fail(STB_ERR_INVALID_ARG, "mesh, V, g and f must be given");
    size_t need;
    stb_status st = stb_assemble_vrhs_workspace_size(mesh, params, nrhs, &need);
    if (st) return st;
    if ((st = check_workspace(ws, ws_bytes, need))) return st;
    const Mesh &m = mesh->m;
    if (m.n_tris > 65535) return fail(STB_ERR_INVALID_ARG, "dense assembly supports E <= 65535");
    AssemblyLayout L = assembly_layout(m, *params, ws, ws_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    if ((st = prepare_mixed(m, *params, L, status_word(ws), s))) return st;
    STB_CUDA(cudaMemsetAsync(f, 0, sizeof(double) * (size_t)nrhs * params->n_steps * m.n_tris, s));
    return run_vrhs_mixed(m, *params, (float *)V, g, nrhs, f, L, s);
}

// ---- non-uniform time grids (Sec. 7) ----------------------------------------
namespace {
struct NuHost {
    std::vector<double> levels;  // [n_levels][LV_STRIDE]
    std::vector<int32_t> off, blk;
    std::vector<double> coef;
    int n_levels = 0;
};

stb_status nu_check(const stb_params *p, const double *times) {
    if (!times) return fail(STB_ERR_INVALID_ARG, "times must be given");
    if (times[0] != 0.0) return fail(STB_ERR_INVALID_ARG, "times[0] must be 0");
    for (int k = 0; k < p->n_steps; ++k)
        if (!(times[k + 1] > times[k]) || !std::isfinite(times[k + 1]))
            return fail(STB_ERR_INVALID_ARG, "times must increase strictly (step %d)", k);
    if (p->n_steps > 256) return fail(STB_ERR_INVALID_ARG, "non-uniform grids support n_steps <= 256");
    return STB_OK;
}

// The distinct time differences and, per difference, the blocks it enters.
NuHost nu_lists(const stb_params &p, const double *t) {
    const int n = p.n_steps;
    std::map<double, int> index;
    index[0.0] = 0;
    std::vector<std::vector<std::pair<int32_t, double>>> per(1);
    std::vector<std::pair<int32_t, double>> sing;
    auto level = [&](double d) {
        auto it = index.find(d);
        if (it != index.end()) return it->second;
        const int L = (int)per.size();
        index[d] = L;
        per.emplace_back();
        return L;
    };
    for (int k = 0; k < n; ++k)
        for (int i = 0; i <= k; ++i) {
            const int32_t b = k * (k + 1) / 2 + i;
            if (i == k) {
                const double h = t[k + 1] - t[k];
                per[level(h)].push_back({b, -1.0});
                per[0].push_back({b, 1.0});
                sing.push_back({b, h});
            } else {
                per[level(t[k + 1] - t[i + 1])].push_back({b, 1.0});
                per[level(t[k] - t[i + 1])].push_back({b, -1.0});
                per[level(t[k + 1] - t[i])].push_back({b, -1.0});
                per[level(t[k] - t[i])].push_back({b, 1.0});
            }
        }
    NuHost H;
    H.n_levels = (int)per.size();
    H.levels.assign((size_t)H.n_levels * LV_STRIDE, 0.0);
    const double pi = 3.14159265358979323846, al = p.alpha;
    for (auto &kv : index) {
        if (kv.second == 0) continue;
        const double delta = kv.first, sd = std::sqrt(delta);
        double *lv = H.levels.data() + (size_t)kv.second * LV_STRIDE;
        lv[LV_C] = 1.0 / (2.0 * std::sqrt(al * delta));
        lv[LV_B] = delta / (4.0 * pi * al);
        lv[LV_CC] = sd / (4.0 * pi * std::sqrt(pi * al * al * al));
        lv[LV_D] = delta / (4.0 * pi);
        lv[LV_E] = sd / (4.0 * pi * std::sqrt(pi * al));
    }
    H.off.push_back(0);
    for (int L = 0; L <= H.n_levels; ++L) {
        const auto &lst = L < H.n_levels ? per[L] : sing;
        for (auto &e : lst) {
            H.blk.push_back(e.first);
            H.coef.push_back(e.second);
        }
        H.off.push_back((int32_t)H.blk.size());
    }
    return H;
}

size_t nu_table_bytes(const NuHost &H) {
    return align256(sizeof(double) * H.levels.size()) + align256(sizeof(int32_t) * H.off.size()) +
           align256(sizeof(int32_t) * H.blk.size()) + align256(sizeof(double) * H.coef.size());
}

// Mixed path: FP32 regular rule, closed-form records, Gauss nodes, targets.
struct NuMixHost {
    std::vector<float> rule, ss, cf, nodes;  // rule and ss: FP32 regular and difference-form rules
    std::vector<int32_t> targets;
};

NuMixHost nu_mixed_host(const stb_params &p, const double *t) {
    NuMixHost M;
    std::vector<float> unodes;
    stb_params pm = p;
    pm.precision = STB_PREC_MIXED;
    mixed_tables(pm, M.rule, M.ss, unodes);
    nu_mixed_tables(p, t, M.cf, M.nodes, M.targets);
    return M;
}

size_t nu_mixed_bytes(const NuMixHost &M) {
    return align256(sizeof(float) * M.rule.size()) + align256(sizeof(float) * M.ss.size()) +
           align256(sizeof(float) * M.cf.size()) + align256(sizeof(float) * M.nodes.size()) +
           align256(sizeof(int32_t) * M.targets.size());
}

size_t nu_mixed_bytes(const stb_params &p, const double *t) {
    return nu_mixed_bytes(nu_mixed_host(p, t));
}
}  // namespace

extern "C" stb_status stb_assemble_nu_mixed_counts(const stb_params *params, const double *times,
                                                   int64_t *closed_form_terms, int64_t *gauss_nodes,
                                                   int64_t *closed_form_blocks) {
    if (!params) return fail(STB_ERR_INVALID_ARG, "params must be given");
    stb_status st = nu_check(params, times);
    if (st) return st;
    stb_params p = *params;
    p.T = times[p.n_steps];
    if ((st = check_assembly_params(&p))) return st;
    std::vector<float> cf, nodes;
    std::vector<int32_t> targets;
    nu_mixed_tables(p, times, cf, nodes, targets);
    int64_t terms = 0, nn = 0, blocks = 0;
    for (size_t r = 0; r < cf.size(); r += NU_CF_FLOATS) {
        int32_t cnt;
        std::memcpy(&cnt, &cf[r + 1], sizeof cnt);
        blocks += cnt >> 1;
        for (int t = 0; t < 4; ++t) terms += cf[r + 7 + 4 * t] != 0.f ? 1 : 0;
    }
    for (size_t q = 0; q < nodes.size(); q += 4) nn += nodes[q + 1] != 0.f || nodes[q] != 0.f ? 1 : 0;
    if (closed_form_terms) *closed_form_terms = terms;
    if (gauss_nodes) *gauss_nodes = nn;
    if (closed_form_blocks) *closed_form_blocks = blocks;
    return STB_OK;
}

extern "C" stb_status stb_assemble_nu_workspace_size(const stb_mesh *mesh, const stb_params *params,
                                                     const double *times, size_t *bytes) {
    if (!mesh || !params || !bytes) return fail(STB_ERR_INVALID_ARG, "mesh, params and bytes must be given");
    stb_status st = nu_check(params, times);
    if (st) return st;
    stb_params p = *params;
    p.T = times[p.n_steps];
    if ((st = check_assembly_params(&p))) return st;
    if (p.storage != STB_STORE_F64)
        return fail(STB_ERR_INVALID_ARG, "non-uniform grids store FP64 blocks (STB_STORE_F64)");
    const bool mixed = p.precision == STB_PREC_MIXED;
    p.precision = STB_PREC_FP64;  // the touching pairs take the FP64 path
    *bytes = align256(assembly_layout(mesh->m, p, nullptr, 0).bytes) + nu_table_bytes(nu_lists(p, times));
    if (mixed) *bytes += nu_mixed_bytes(p, times);
    return STB_OK;
}

extern "C" stb_status stb_assemble_nu(const stb_mesh *mesh, const stb_params *params,
                                      const double *times, double *V, double *K, void *ws,
                                      size_t ws_bytes, stb_stream stream) {
    if (!V || !K) return fail(STB_ERR_INVALID_ARG, "V and K must be given");
    size_t need;
    stb_status st = stb_assemble_nu_workspace_size(mesh, params, times, &need);
    if (st) return st;
    if ((st = check_workspace(ws, ws_bytes, need))) return st;
    const Mesh &m = mesh->m;
    if (m.n_tris > 65535) return fail(STB_ERR_INVALID_ARG, "dense assembly supports E <= 65535");
    stb_params p = *params;
    p.T = times[p.n_steps];
    const bool mixed = p.precision == STB_PREC_MIXED;
    p.precision = STB_PREC_FP64;  // layout and tables of the FP64 kernels
    const NuHost H = nu_lists(p, times);
    AssemblyLayout L = assembly_layout(m, p, ws, ws_bytes);
    char *q = static_cast<char *>(ws) + align256(L.bytes);
    double *d_lv = reinterpret_cast<double *>(q);
    q += align256(sizeof(double) * H.levels.size());
    int32_t *d_off = reinterpret_cast<int32_t *>(q);
    q += align256(sizeof(int32_t) * H.off.size());
    int32_t *d_blk = reinterpret_cast<int32_t *>(q);
    q += align256(sizeof(int32_t) * H.blk.size());
    double *d_coef = reinterpret_cast<double *>(q);
    q += align256(sizeof(double) * H.coef.size());
    NuMixHost M;
    float *d_mrule = nullptr, *d_mss = nullptr, *d_cf = nullptr, *d_nodes = nullptr;
    int32_t *d_targets = nullptr;
    if (mixed) {
        M = nu_mixed_host(p, times);
        d_mrule = reinterpret_cast<float *>(q);
        q += align256(sizeof(float) * M.rule.size());
        d_mss = reinterpret_cast<float *>(q);
        q += align256(sizeof(float) * M.ss.size());
        d_cf = reinterpret_cast<float *>(q);
        q += align256(sizeof(float) * M.cf.size());
        d_nodes = reinterpret_cast<float *>(q);
        q += align256(sizeof(float) * M.nodes.size());
        d_targets = reinterpret_cast<int32_t *>(q);
    }
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    if ((st = prepare_fp64(m, p, L, status_word(ws), s))) return st;
    STB_CUDA(cudaMemcpyAsync(d_lv, H.levels.data(), sizeof(double) * H.levels.size(),
                             cudaMemcpyHostToDevice, s));
    STB_CUDA(cudaMemcpyAsync(d_off, H.off.data(), sizeof(int32_t) * H.off.size(),
                             cudaMemcpyHostToDevice, s));
    STB_CUDA(cudaMemcpyAsync(d_blk, H.blk.data(), sizeof(int32_t) * H.blk.size(),
                             cudaMemcpyHostToDevice, s));
    STB_CUDA(cudaMemcpyAsync(d_coef, H.coef.data(), sizeof(double) * H.coef.size(),
                             cudaMemcpyHostToDevice, s));
    const int E = (int)m.n_tris;
    const size_t nblk = (size_t)p.n_steps * (p.n_steps + 1) / 2;
    STB_CUDA(cudaMemsetAsync(V, 0, sizeof(double) * nblk * E * E, s));
    STB_CUDA(cudaMemsetAsync(K, 0, sizeof(double) * nblk * E * E, s));
    NuLists lists{d_lv, d_off, d_blk, d_coef, H.n_levels};
    Globals g = make_globals(p);
    if (mixed) {
        auto up = [&](void *dst, const void *src, size_t bytes) {
            return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
        };
        STB_CUDA(up(d_mrule, M.rule.data(), sizeof(float) * M.rule.size()));
        STB_CUDA(up(d_mss, M.ss.data(), sizeof(float) * M.ss.size()));
        STB_CUDA(up(d_cf, M.cf.data(), sizeof(float) * M.cf.size()));
        STB_CUDA(up(d_nodes, M.nodes.data(), sizeof(float) * M.nodes.size()));
        STB_CUDA(up(d_targets, M.targets.data(), sizeof(int32_t) * M.targets.size()));
        // the host tables are pageable: the copies have been staged when the
        // calls return, so M may go out of scope afterwards
        if ((st = run_nu_regular_mixed(m, p, L.geo, d_mrule, d_cf,
                                       (int)(M.cf.size() / NU_CF_FLOATS), d_nodes,
                                       (int)(M.nodes.size() / 4), d_targets, V, K, s)))
            return st;
        const int ss_n[4] = {0, (int)L.ss_n[1], (int)L.ss_n[2], (int)L.ss_n[3]};
        return run_nu_singular_mixed(m, p, L.geo, L.pairs, d_mss, ss_n, d_cf,
                                     (int)(M.cf.size() / NU_CF_FLOATS), d_nodes,
                                     (int)(M.nodes.size() / 4), d_targets, V, K, s);
    } else {
        dim3 grid((E + REG_THREADS - 1) / REG_THREADS, E);
        count_launch(s);
        k_regular_nu_f64<4><<<grid, REG_THREADS, 0, s>>>(L.geo, m.d_tris, E, L.rule,
                                                         p.quad_regular * p.quad_regular, lists, g,
                                                         V, K);
        if ((st = check_launch("k_regular_nu_f64"))) return st;
    }
    if (m.n_touch == 0) return STB_OK;
    SSTables tab{};
    const double *base = L.ss;
    for (int cls = 1; cls <= 3; ++cls) {
        size_t n = L.ss_n[cls];
        tab.s1[cls] = base;
        tab.s2[cls] = base + n;
        tab.t1[cls] = base + 2 * n;
        tab.t2[cls] = base + 3 * n;
        tab.w[cls] = base + 4 * n;
        tab.n[cls] = (int)n;
        base += 5 * n;
    }
    count_launch(s);
    k_singular_nu_f64<4><<<(unsigned)m.n_touch, SS_THREADS, 0, s>>>(L.geo, L.pairs, E, tab, lists,
                                                                    g, V, K);
    return check_launch("k_singular_nu_f64");
}

