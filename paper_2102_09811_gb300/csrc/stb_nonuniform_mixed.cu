// stb_nonuniform_mixed.cu -- mixed-precision separated-pair assembly of V
// and K on a non-uniform time grid (Sec. 7: the antiderivatives carry over
// to arbitrary steps); every quadrature point in FP32, blocks stored FP64.
//
// Block (k, i) of the packed layout (b = k (k + 1) / 2 + i) is, for fixed
// r = x - y, the time integral
//   A^{k,i}(r) = int omega_{k,i}(delta) G(r, delta) d delta      (K: G -> (r.n_y) / (2 delta) G),
// omega_{k,i}(delta) = |I_k cap (I_i + delta)|, the overlap of the trial
// interval shifted by delta with the test interval: for k > i a trapezoid on
// [a, a + h_k + h_i], a = t_k - t_{i+1}, rising on [a, a + min(h_k, h_i)],
// flat up to a + max(h_k, h_i) and falling to zero; for k = i the ramp
// h_k - delta on [0, h_k].  As on the uniform grid, nothing is differenced
// where FP32 would cancel:
//  * k = i and k = i + 1 (the weight reaches delta = 0): closed forms over
//    corner differences,  sum_t sigma_t H(delta_t)  with H the closed form
//    of the uniform path's block 0 (and its K counterpart): k = i: H(h_k);
//    k = i + 1 with the shorter step B and the longer A: the hat of two
//    steps B, -2 H(B) + H(2 B) (the uniform block 1, well conditioned), and
//    the rest of the trapezoid, omega - hat = the overlap weight of steps
//    A - B and B at gap B, by Gauss nodes added to it (A = B: nothing
//    added; -H(A) + H(A + B) - H(B) directly would difference terms of
//    size A where the block is of size B).  The corners annihilate the
//    part linear in delta, left out where x = rho / (2 sqrt(alpha delta_max)) < 1;
//  * k >= i + 2 (a > 0): Gauss-Legendre on the pieces of the trapezoid,
//    each piece cut at 2 p0, 4 p0, ... until every part starts at least its
//    own length away from delta = 0, with 6, 4, 3 or 2 nodes by that ratio
//    (the counts of the uniform path's intervals k = 1, k >= 2, k >= 16,
//    k >= 96).  A closed form over four corners at a small positive gap
//    would difference four terms of like size in FP32; the cut pieces keep
//    every node away from the steep start of the kernel instead.
// Blocks with the same differences (up to 2^-44 T) share their evaluation:
// on a uniform grid there are two closed forms and one node list per block
// distance d >= 2.  Touching pairs come from the FP64 kernel afterwards.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "stb_assemble.h"
#include "stb_mixed_math.h"

namespace stb {

constexpr int NU_THREADS = 128;
constexpr int NU_MAX_RULE = 256;
constexpr int NU_CFC = 4;   // closed-form records per pass over the points
constexpr int NU_NG = 32;   // Gauss nodes per pass over the points
// node tag of the last node of a list: (target offset << 10) | (add << 9) |
// target count; add: the list completes a block whose closed-form part is
// already stored
constexpr int NU_TAG_BITS = 10, NU_ADD_BIT = 9, NU_CNT_MASK = (1 << NU_ADD_BIT) - 1;

namespace {

float int_bits(int32_t v) {
    float f;
    std::memcpy(&f, &v, sizeof f);
    return f;
}

int gauss_count(double ratio) {
    return ratio < 2.0 ? 6 : ratio < 16.0 ? 4 : ratio < 96.0 ? 3 : 2;
}

}  // namespace

// Host tables of the mixed non-uniform path: closed-form records
// (NU_CF_FLOATS floats each, padded to NU_CFC records), Gauss nodes (float4
// (b, cV, cK, tag), padded to NU_NG) and the target blocks of both.
void nu_mixed_tables(const stb_params &p, const double *t, std::vector<float> &cf,
                     std::vector<float> &nodes, std::vector<int32_t> &targets) {
    const double pi = 3.14159265358979323846, al = p.alpha, log2e = 1.4426950408889634;
    const int n = p.n_steps;
    const double T = t[n];
    auto key = [&](double x) { return (long long)std::llround(x / T * 17592186044416.0); };
    // (form, differences): 0 diagonal closed form, 3 closed form of the hat at
    // k = i + 1, 1 node list of a gap a > 0, 2 node list added to a form-3 block
    using Key = std::tuple<int, long long, long long, long long>;
    std::map<Key, std::vector<int32_t>> cf_map, g_map;
    std::map<Key, std::tuple<double, double, double>> args;
    for (int k = 0; k < n; ++k)
        for (int i = 0; i <= k; ++i) {
            const int32_t b = k * (k + 1) / 2 + i;
            const double hk = t[k + 1] - t[k], hi = t[i + 1] - t[i];
            const double a = i == k ? 0.0 : t[k] - t[i + 1];
            if (i == k) {
                const Key kk{0, key(hk), 0, 0};
                cf_map[kk].push_back(b);
                args[kk] = {0.0, hk, hk};
            } else if (a > 0.0) {  // k >= i + 2
                const Key kk{1, key(a), key(hk), key(hi)};
                g_map[kk].push_back(b);
                args[kk] = {a, hk, hi};
            } else {  // k = i + 1: the hat of the shorter step B, plus the rest
                const double B = std::min(hk, hi), A = std::max(hk, hi);
                const Key kc{3, 0, key(B), key(B)};  // own type: no key shared with a node list
                cf_map[kc].push_back(b);
                args[kc] = {0.0, B, B};
                if (key(A) != key(B)) {
                    const Key kg{2, key(B), key(A - B), key(B)};
                    g_map[kg].push_back(b);
                    args[kg] = {B, A - B, B};
                }
            }
        }
    cf.clear();
    nodes.clear();
    targets.clear();
    for (auto &kv : cf_map) {
        const auto [a, hk, hi] = args[kv.first];
        const bool diag = std::get<0>(kv.first) == 0;
        double dl[4], sg[4];
        int nt;
        if (diag) {
            dl[0] = hk;
            sg[0] = 1.0;
            nt = 1;
        } else {
            dl[0] = a + hk;       // t_{k+1} - t_{i+1}
            dl[1] = a;            // t_k - t_{i+1}
            dl[2] = a + hk + hi;  // t_{k+1} - t_i
            dl[3] = a + hi;       // t_k - t_i
            sg[0] = -1.0, sg[1] = 1.0, sg[2] = 1.0, sg[3] = -1.0;
            nt = 4;
        }
        float rec[NU_CF_FLOATS] = {};
        double dmax = 0.0, kconst = 0.0;
        int m = 0;
        for (int u = 0; u < nt; ++u) {
            if (dl[u] <= 0.0) {  // H(0) = 0; psi(infinity) = 1/2
                kconst += 0.5 * sg[u];
                continue;
            }
            dmax = std::max(dmax, dl[u]);
            rec[4 + 4 * m] = (float)(1.0 / (2.0 * std::sqrt(al * dl[u])));
            rec[5 + 4 * m] = (float)(2.0 * std::sqrt(al * dl[u]));
            rec[6 + 4 * m] = (float)(std::sqrt(dl[u]) / (4.0 * pi * std::pow(al, 1.5)));
            rec[7 + 4 * m] = (float)sg[u];
            ++m;
        }
        for (; m < 4; ++m) {
            rec[4 + 4 * m] = 1.f;
            rec[5 + 4 * m] = 1.f;
        }
        rec[0] = int_bits((int32_t)targets.size());
        rec[1] = int_bits(((int32_t)kv.second.size() << 1) | (diag ? 0 : 1));
        rec[2] = (float)(1.0 / (2.0 * std::sqrt(al * dmax)));
        rec[3] = (float)kconst;
        targets.insert(targets.end(), kv.second.begin(), kv.second.end());
        cf.insert(cf.end(), rec, rec + NU_CF_FLOATS);
    }
    while (cf.size() % (NU_CFC * NU_CF_FLOATS)) {  // records without targets
        float rec[NU_CF_FLOATS] = {};
        rec[0] = int_bits(0);
        rec[1] = int_bits(0);
        rec[2] = 1.f;
        for (int m = 0; m < 4; ++m) rec[4 + 4 * m] = rec[5 + 4 * m] = 1.f;
        cf.insert(cf.end(), rec, rec + NU_CF_FLOATS);
    }
    std::vector<double> u, w;
    for (auto &kv : g_map) {
        const auto [a, hk, hi] = args[kv.first];
        const double hmin = std::min(hk, hi), hmax = std::max(hk, hi), b = a + hk + hi;
        // one linear piece of the trapezoid: omega(delta) = c0 + c1 delta on [p0, p1]
        auto piece = [&](double p0, double p1, double c0, double c1) {
            while (p0 < p1) {
                const double q1 = p1 - p0 > p0 ? 2.0 * p0 : p1, L = q1 - p0;
                const int ng = gauss_count(p0 / L);
                u.resize(ng);
                w.resize(ng);
                gauss_legendre01(ng, u.data(), w.data());
                for (int q = 0; q < ng; ++q) {
                    const double delta = p0 + L * u[q];
                    const double cv = L * w[q] * (c0 + c1 * delta) * std::pow(4.0 * pi * al * delta, -1.5);
                    nodes.push_back((float)(-log2e / (4.0 * al * delta)));
                    nodes.push_back((float)cv);
                    nodes.push_back((float)(cv / (2.0 * delta)));
                    nodes.push_back(int_bits(-1));
                }
                p0 = q1;
            }
        };
        piece(a, a + hmin, -a, 1.0);
        if (hmax > hmin) piece(a + hmin, a + hmax, hmin, 0.0);
        piece(a + hmax, b, b, -1.0);
        const int32_t cnt = (int32_t)kv.second.size(), add = std::get<0>(kv.first) == 2;
        nodes.back() = int_bits(((int32_t)targets.size() << NU_TAG_BITS) | (add << NU_ADD_BIT) | cnt);
        targets.insert(targets.end(), kv.second.begin(), kv.second.end());
    }
    while (nodes.size() % (4 * NU_NG)) {  // zero nodes, no target
        nodes.push_back(0.f);
        nodes.push_back(0.f);
        nodes.push_back(0.f);
        nodes.push_back(int_bits(-1));
    }
    if (targets.empty()) targets.push_back(0);
}

// All closed-form and Gauss blocks of the separated pair (l, j) of one CTA
// row l; threads whose pair touches or lies past E only join the barriers
// of the shared table chunks.
__global__ void __launch_bounds__(NU_THREADS)
k_regular_nu_mixed(const double *__restrict__ geo, const int32_t *__restrict__ tris, int E,
                   const float *__restrict__ rule, int nq, const float *__restrict__ cf, int n_cf,
                   const float4 *__restrict__ nodes, int n_nodes,
                   const int32_t *__restrict__ targets, float pK, double *__restrict__ V,
                   double *__restrict__ K) {
    __shared__ float4 xa[NU_MAX_RULE];
    __shared__ __align__(16) float s_cf[NU_CFC * NU_CF_FLOATS];
    __shared__ __align__(16) float s_b[NU_NG];
    __shared__ float s_cv[NU_NG], s_ck[NU_NG];
    __shared__ int s_tag[NU_NG];
    const int l = blockIdx.y;
    const int j = blockIdx.x * NU_THREADS + threadIdx.x;
    const double *gl = geo + (size_t)l * GEO_STRIDE;
    for (int a = threadIdx.x; a < nq; a += NU_THREADS) {  // x_a - P0_l and w_a
        const double s1 = rule[4 * a], s2 = rule[4 * a + 1];
        double pt[3];
        for (int c = 0; c < 3; ++c)
            pt[c] = s1 * (gl[GEO_V1 + c] - gl[GEO_V0 + c]) + s2 * (gl[GEO_V2 + c] - gl[GEO_V1 + c]);
        xa[a] = make_float4((float)pt[0], (float)pt[1], (float)pt[2], rule[4 * a + 2]);
    }
    bool active = j < E;
    float D[3] = {0.f, 0.f, 0.f}, B1[3] = {0.f, 0.f, 0.f}, B2[3] = {0.f, 0.f, 0.f},
          nv[3] = {0.f, 0.f, 0.f}, scale = 0.f;
    if (active) {
        const int32_t tl[3] = {tris[3 * l], tris[3 * l + 1], tris[3 * l + 2]};
        const int32_t tj[3] = {tris[3 * j], tris[3 * j + 1], tris[3 * j + 2]};
        for (int i = 0; i < 3; ++i)
            if (tl[i] == tj[0] || tl[i] == tj[1] || tl[i] == tj[2]) active = false;
        const double *gj = geo + (size_t)j * GEO_STRIDE;
        for (int c = 0; c < 3; ++c) {
            D[c] = (float)(gl[GEO_V0 + c] - gj[GEO_V0 + c]);
            B1[c] = (float)(gj[GEO_V1 + c] - gj[GEO_V0 + c]);
            B2[c] = (float)(gj[GEO_V2 + c] - gj[GEO_V1 + c]);
            nv[c] = (float)gj[GEO_N + c];
        }
        scale = (float)(4.0 * gl[GEO_AREA] * gj[GEO_AREA]);
    }
    const size_t EE = (size_t)E * E, ij = (size_t)l * E + j;

    // closed forms, NU_CFC records per pass over the points
    for (int c0 = 0; c0 < n_cf; c0 += NU_CFC) {
        __syncthreads();
        for (int i = threadIdx.x; i < NU_CFC * NU_CF_FLOATS; i += NU_THREADS)
            s_cf[i] = cf[(size_t)c0 * NU_CF_FLOATS + i];
        __syncthreads();
        if (!active) continue;
        float av[NU_CFC], ak[NU_CFC];
#pragma unroll
        for (int u = 0; u < NU_CFC; ++u) av[u] = ak[u] = 0.f;
        for (int b = 0; b < nq; ++b) {
            const float t1 = rule[4 * b], t2 = rule[4 * b + 1], wb = rule[4 * b + 2];
            const float r0b = D[0] - (t1 * B1[0] + t2 * B2[0]);
            const float r1b = D[1] - (t1 * B1[1] + t2 * B2[1]);
            const float r2b = D[2] - (t1 * B1[2] + t2 * B2[2]);
            for (int a = 0; a < nq; ++a) {
                const float4 xq = xa[a];
                const float r0 = r0b + xq.x, r1 = r1b + xq.y, r2 = r2b + xq.z;
                const float rr = r0 * r0 + r1 * r1 + r2 * r2;
                const float irho = rsqrtf(rr), rho = rr * irho;
                const float w = xq.w * wb;
                const float wrk = w * (r0 * nv[0] + r1 * nv[1] + r2 * nv[2]) * irho;
#pragma unroll
                for (int u = 0; u < NU_CFC; ++u) {
                    const float *rec = s_cf + u * NU_CF_FLOATS;
                    const float4 hd = ld_tab<true>(rec);
                    const bool small = (__float_as_int(hd.y) & 1) && rho * hd.z < 1.f;
                    float hv = 0.f, qk = small ? hd.w : 0.f;
#pragma unroll
                    for (int tt = 0; tt < 4; ++tt) {
                        const float4 tm = ld_tab<true>(rec + 4 + 4 * tt);  // c, 1/c, pV, sigma
                        if (tm.w == 0.f) continue;
                        const float x = rho * tm.x, ix = irho * tm.y;
                        const float ec = erfcf(x), ee = expf(-x * x);
                        if (small) {
                            const float ef = erff(x);
                            hv = fmaf(tm.w * tm.z, x * ec - 0.5f * ef * ix - ee * ISQRTPI, hv);
                            qk = fmaf(tm.w, psi32(x, ix, ef, ee), qk);
                        } else {
                            hv = fmaf(tm.w * tm.z, (x + 0.5f * ix) * ec - ee * ISQRTPI, hv);
                            qk = fmaf(tm.w, ec * (0.25f * ix * ix - 0.5f) + 0.5f * ISQRTPI * ee * ix, qk);
                        }
                    }
                    av[u] = fmaf(w, hv, av[u]);
                    ak[u] = fmaf(wrk, qk, ak[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < NU_CFC; ++u) {
            const int off = __float_as_int(s_cf[u * NU_CF_FLOATS]);
            const int cnt = __float_as_int(s_cf[u * NU_CF_FLOATS + 1]) >> 1;
            for (int e = 0; e < cnt; ++e) {
                const size_t o = (size_t)targets[off + e] * EE + ij;
                V[o] = (double)(scale * av[u]);
                K[o] = (double)(scale * pK * ak[u]);
            }
        }
    }

    // Gauss nodes, NU_NG per pass: points contracted per node first, then
    // the node weights applied in order; the last node of a node list
    // stores its blocks
    float runV = 0.f, runK = 0.f;
    for (int q0 = 0; q0 < n_nodes; q0 += NU_NG) {
        __syncthreads();
        if (threadIdx.x < NU_NG) {
            const float4 nd = nodes[q0 + threadIdx.x];
            s_b[threadIdx.x] = nd.x;
            s_cv[threadIdx.x] = nd.y;
            s_ck[threadIdx.x] = nd.z;
            s_tag[threadIdx.x] = __float_as_int(nd.w);
        }
        __syncthreads();
        if (!active) continue;
        float2 Es[NU_NG / 4][2], Fs[NU_NG / 4][2];
#pragma unroll
        for (int g = 0; g < NU_NG / 4; ++g) Es[g][0] = Es[g][1] = Fs[g][0] = Fs[g][1] = make_float2(0.f, 0.f);
        for (int b = 0; b < nq; ++b) {
            const float t1 = rule[4 * b], t2 = rule[4 * b + 1], wb = rule[4 * b + 2];
            const float r0b = D[0] - (t1 * B1[0] + t2 * B2[0]);
            const float r1b = D[1] - (t1 * B1[1] + t2 * B2[1]);
            const float r2b = D[2] - (t1 * B1[2] + t2 * B2[2]);
            for (int a = 0; a < nq; ++a) {
                const float4 xq = xa[a];
                const float r0 = r0b + xq.x, r1 = r1b + xq.y, r2 = r2b + xq.z;
                const float rr = r0 * r0 + r1 * r1 + r2 * r2;
                const float w = xq.w * wb, wrn = w * (r0 * nv[0] + r1 * nv[1] + r2 * nv[2]);
                const float2 rr2 = make_float2(rr, rr), w2 = make_float2(w, w), wrn2 = make_float2(wrn, wrn);
#pragma unroll
                for (int g = 0; g < NU_NG / 4; ++g) {
                    const float4 bq = ld_tab<true>(s_b + 4 * g);
                    const float2 t01 = __fmul2_rn(rr2, make_float2(bq.x, bq.y));
                    const float2 t23 = __fmul2_rn(rr2, make_float2(bq.z, bq.w));
                    const float2 e01 = make_float2(ex2(t01.x), ex2(t01.y));
                    const float2 e23 = make_float2(ex2(t23.x), ex2(t23.y));
                    Es[g][0] = __ffma2_rn(w2, e01, Es[g][0]);
                    Fs[g][0] = __ffma2_rn(wrn2, e01, Fs[g][0]);
                    Es[g][1] = __ffma2_rn(w2, e23, Es[g][1]);
                    Fs[g][1] = __ffma2_rn(wrn2, e23, Fs[g][1]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NU_NG; ++q) {
            const float2 ep = Es[q >> 2][(q >> 1) & 1], fp = Fs[q >> 2][(q >> 1) & 1];
            runV = fmaf(s_cv[q], (q & 1) ? ep.y : ep.x, runV);
            runK = fmaf(s_ck[q], (q & 1) ? fp.y : fp.x, runK);
            const int tag = s_tag[q];
            if (tag >= 0) {
                const int off = tag >> NU_TAG_BITS, cnt = tag & NU_CNT_MASK;
                const bool add = (tag >> NU_ADD_BIT) & 1;
                for (int e = 0; e < cnt; ++e) {
                    const size_t o = (size_t)targets[off + e] * EE + ij;
                    // add: the closed-form part of this block was stored by
                    // this thread in the first phase
                    V[o] = (add ? V[o] : 0.0) + (double)(scale * runV);
                    K[o] = (add ? K[o] : 0.0) + (double)(scale * runK);
                }
                runV = runK = 0.f;
            }
        }
    }
}

// ----------------------------------------------------------- touching pairs ---
constexpr int NU_SS_THREADS = 128;
constexpr int NU_SS_NG = 16;  // Gauss nodes per pass over the regularised rule

// One closed-form record at one point: hv (V) and qk (K / (r.n_y) without
// the 1/(4 pi alpha rho) factor), as in the separated-pair kernel.
__device__ __forceinline__ void nu_cf_point(const float *rec, float rho, float irho, float &hv,
                                            float &qk) {
    const float4 hd = ld_tab<true>(rec);
    const bool small = (__float_as_int(hd.y) & 1) && rho * hd.z < 1.f;
    hv = 0.f;
    qk = small ? hd.w : 0.f;
#pragma unroll
    for (int tt = 0; tt < 4; ++tt) {
        const float4 tm = ld_tab<true>(rec + 4 + 4 * tt);  // c, 1/c, pV, sigma
        if (tm.w == 0.f) continue;
        const float x = rho * tm.x, ix = irho * tm.y;
        const float ec = erfcf(x), ee = expf(-x * x);
        if (small) {
            const float ef = erff(x);
            hv = fmaf(tm.w * tm.z, x * ec - 0.5f * ef * ix - ee * ISQRTPI, hv);
            qk = fmaf(tm.w, psi32(x, ix, ef, ee), qk);
        } else {
            hv = fmaf(tm.w * tm.z, (x + 0.5f * ix) * ec - ee * ISQRTPI, hv);
            qk = fmaf(tm.w, ec * (0.25f * ix * ix - 0.5f) + 0.5f * ISQRTPI * ee * ix, qk);
        }
    }
}

// All blocks of the touching pair P, both orders (entry (a,b): r = x - y and
// n_b; entry (b,a): -r and n_a), from the regularised rules in difference
// form (x - y = p0 X0 + p1 X1 + p2 X2 + p3 X3 per class, FP32 tables mss:
// per class p0, p1, p2, p3, w of n[cls] points); one CTA per pair, the
// point sums reduced over the CTA.  Identical pairs: K = 0 (flat triangle).
__global__ void __launch_bounds__(NU_SS_THREADS)
k_singular_nu_mixed(const double *__restrict__ geo, const TouchPair *__restrict__ pairs, int E,
                    const float *__restrict__ mss, int n1, int n2, int n3,
                    const float *__restrict__ cf, int n_cf, const float4 *__restrict__ nodes,
                    int n_nodes, const int32_t *__restrict__ targets, float pK,
                    double *__restrict__ V, double *__restrict__ K) {
    __shared__ float red[NU_SS_THREADS / 32][3 * NU_SS_NG];
    __shared__ float fin[3 * NU_SS_NG];
    __shared__ __align__(16) float s_cf[NU_CFC * NU_CF_FLOATS];
    __shared__ __align__(16) float s_b[NU_SS_NG];
    __shared__ float s_cv[NU_SS_NG], s_ck[NU_SS_NG];
    __shared__ int s_tag[NU_SS_NG];
    const TouchPair P = pairs[blockIdx.x];
    const int a = P.a, b = P.b, cls = P.cls;
    if (a < 0 || b < a || b >= E || cls < PAIR_VERTEX || cls > PAIR_IDENTICAL) return;
    const double *ga = geo + (size_t)a * GEO_STRIDE, *gb = geo + (size_t)b * GEO_STRIDE;
    float X[4][3], na[3], nb[3];
    {
        const int oa0 = P.perm & 3, oa1 = (P.perm >> 2) & 3, oa2 = (P.perm >> 4) & 3;
        const int ob0 = (P.perm >> 6) & 3, ob1 = (P.perm >> 8) & 3, ob2 = (P.perm >> 10) & 3;
        for (int c = 0; c < 3; ++c) {
            const double A1 = ga[3 * oa1 + c] - ga[3 * oa0 + c], A2 = ga[3 * oa2 + c] - ga[3 * oa1 + c];
            const double Bv1 = gb[3 * ob1 + c] - gb[3 * ob0 + c], Bv2 = gb[3 * ob2 + c] - gb[3 * ob1 + c];
            if (cls == PAIR_IDENTICAL) {
                X[0][c] = (float)-A1; X[1][c] = (float)-A2; X[2][c] = 0.f; X[3][c] = 0.f;
            } else if (cls == PAIR_EDGE) {
                X[0][c] = (float)-A1; X[1][c] = (float)A2; X[2][c] = (float)-Bv2; X[3][c] = 0.f;
            } else {
                X[0][c] = (float)A1; X[1][c] = (float)A2; X[2][c] = (float)-Bv1; X[3][c] = (float)-Bv2;
            }
            na[c] = (float)ga[GEO_N + c];
            nb[c] = (float)gb[GEO_N + c];
        }
    }
    const double scale = 4.0 * ga[GEO_AREA] * gb[GEO_AREA];
    const bool ident = cls == PAIR_IDENTICAL;
    const int npt = cls == PAIR_VERTEX ? n1 : cls == PAIR_EDGE ? n2 : n3;
    const float *base = mss + (cls >= PAIR_EDGE ? 5 * (size_t)n1 : 0) + (cls == PAIR_IDENTICAL ? 5 * (size_t)n2 : 0);
    const float *R0 = base, *R1 = base + npt, *R2 = base + 2 * (size_t)npt,
                *R3 = base + 3 * (size_t)npt, *W = base + 4 * (size_t)npt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t EE = (size_t)E * E, iab = (size_t)a * E + b, iba = (size_t)b * E + a;
    auto point = [&](int p, float &rr, float &rab, float &rba, float &w) {
        const float q0 = R0[p], q1 = R1[p], q2 = R2[p], q3 = R3[p];
        float r[3];
        for (int c = 0; c < 3; ++c) r[c] = q0 * X[0][c] + q1 * X[1][c] + q2 * X[2][c] + q3 * X[3][c];
        rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        rab = r[0] * nb[0] + r[1] * nb[1] + r[2] * nb[2];
        rba = -(r[0] * na[0] + r[1] * na[1] + r[2] * na[2]);
        w = W[p];
    };
    // sums over the CTA of vals[0..nv), into fin (nv <= 3 NU_SS_NG)
    auto reduce = [&](float *vals, int nv) {
        for (int k = 0; k < nv; ++k) {
            float v = vals[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < nv) {
            float t = 0.f;
            for (int wi = 0; wi < NU_SS_THREADS / 32; ++wi) t += red[wi][threadIdx.x];
            fin[threadIdx.x] = t;
        }
        __syncthreads();
    };
    // add: completes a block whose closed-form part thread 0 stored earlier
    auto emit = [&](int off, int cnt, bool add, double v, double ka, double kb) {
        for (int e = 0; e < cnt; ++e) {
            const size_t o = (size_t)targets[off + e] * EE;
            V[o + iab] = (add ? V[o + iab] : 0.0) + v;
            K[o + iab] = ident ? 0.0 : (add ? K[o + iab] : 0.0) + ka;
            if (!ident) {
                V[o + iba] = (add ? V[o + iba] : 0.0) + v;
                K[o + iba] = (add ? K[o + iba] : 0.0) + kb;
            }
        }
    };

    // closed forms
    for (int c0 = 0; c0 < n_cf; c0 += NU_CFC) {
        for (int i = threadIdx.x; i < NU_CFC * NU_CF_FLOATS; i += NU_SS_THREADS)
            s_cf[i] = cf[(size_t)c0 * NU_CF_FLOATS + i];
        __syncthreads();
        float z[3 * NU_CFC];
#pragma unroll
        for (int i = 0; i < 3 * NU_CFC; ++i) z[i] = 0.f;
        for (int p = threadIdx.x; p < npt; p += NU_SS_THREADS) {
            float rr, rab, rba, w;
            point(p, rr, rab, rba, w);
            const float irho = rsqrtf(rr), rho = rr * irho;
#pragma unroll
            for (int u = 0; u < NU_CFC; ++u) {
                float hv, qk;
                nu_cf_point(s_cf + u * NU_CF_FLOATS, rho, irho, hv, qk);
                z[u] = fmaf(w, hv, z[u]);
                z[NU_CFC + u] = fmaf(w * rab * irho, qk, z[NU_CFC + u]);
                z[2 * NU_CFC + u] = fmaf(w * rba * irho, qk, z[2 * NU_CFC + u]);
            }
        }
        reduce(z, 3 * NU_CFC);
        if (threadIdx.x == 0)
            for (int u = 0; u < NU_CFC; ++u)
                emit(__float_as_int(s_cf[u * NU_CF_FLOATS]), __float_as_int(s_cf[u * NU_CF_FLOATS + 1]) >> 1,
                     false, scale * fin[u], scale * pK * fin[NU_CFC + u], scale * pK * fin[2 * NU_CFC + u]);
        __syncthreads();
    }

    // Gauss nodes; thread 0 applies the node weights and stores
    float runV = 0.f, runA = 0.f, runB = 0.f;
    for (int q0 = 0; q0 < n_nodes; q0 += NU_SS_NG) {
        if (threadIdx.x < NU_SS_NG) {
            const float4 nd = nodes[q0 + threadIdx.x];
            s_b[threadIdx.x] = nd.x;
            s_cv[threadIdx.x] = nd.y;
            s_ck[threadIdx.x] = nd.z;
            s_tag[threadIdx.x] = __float_as_int(nd.w);
        }
        __syncthreads();
        float z[3 * NU_SS_NG];
#pragma unroll
        for (int i = 0; i < 3 * NU_SS_NG; ++i) z[i] = 0.f;
        for (int p = threadIdx.x; p < npt; p += NU_SS_THREADS) {
            float rr, rab, rba, w;
            point(p, rr, rab, rba, w);
            const float wa = w * rab, wb = w * rba;
#pragma unroll
            for (int g = 0; g < NU_SS_NG / 4; ++g) {
                const float4 bq = ld_tab<true>(s_b + 4 * g);
                const float e[4] = {ex2(rr * bq.x), ex2(rr * bq.y), ex2(rr * bq.z), ex2(rr * bq.w)};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    z[4 * g + q] = fmaf(w, e[q], z[4 * g + q]);
                    z[NU_SS_NG + 4 * g + q] = fmaf(wa, e[q], z[NU_SS_NG + 4 * g + q]);
                    z[2 * NU_SS_NG + 4 * g + q] = fmaf(wb, e[q], z[2 * NU_SS_NG + 4 * g + q]);
                }
            }
        }
        reduce(z, 3 * NU_SS_NG);
        if (threadIdx.x == 0) {
            for (int q = 0; q < NU_SS_NG; ++q) {
                runV = fmaf(s_cv[q], fin[q], runV);
                runA = fmaf(s_ck[q], fin[NU_SS_NG + q], runA);
                runB = fmaf(s_ck[q], fin[2 * NU_SS_NG + q], runB);
                const int tag = s_tag[q];
                if (tag >= 0) {
                    emit(tag >> NU_TAG_BITS, tag & NU_CNT_MASK, (tag >> NU_ADD_BIT) & 1, scale * runV,
                         scale * runA, scale * runB);
                    runV = runA = runB = 0.f;
                }
            }
        }
        __syncthreads();
    }
}

stb_status run_nu_singular_mixed(const Mesh &m, const stb_params &p, const double *geo,
                                 const TouchPair *pairs, const float *mss, const int (&ss_n)[4],
                                 const float *d_cf, int n_cf, const float *d_nodes, int n_nodes,
                                 const int32_t *d_targets, double *V, double *K, cudaStream_t s) {
    if (m.n_touch == 0) return STB_OK;
    const double pi = 3.14159265358979323846;
    count_launch(s);
    k_singular_nu_mixed<<<(unsigned)m.n_touch, NU_SS_THREADS, 0, s>>>(
        geo, pairs, (int)m.n_tris, mss, ss_n[1], ss_n[2], ss_n[3], d_cf, n_cf,
        reinterpret_cast<const float4 *>(d_nodes), n_nodes, d_targets,
        (float)(1.0 / (4.0 * pi * p.alpha)), V, K);
    return check_launch("k_singular_nu_mixed");
}

stb_status run_nu_regular_mixed(const Mesh &m, const stb_params &p, const double *geo,
                                const float *mrule, const float *d_cf, int n_cf,
                                const float *d_nodes, int n_nodes, const int32_t *d_targets,
                                double *V, double *K, cudaStream_t s) {
    const int E = (int)m.n_tris, nq = p.quad_regular * p.quad_regular;
    if (nq > NU_MAX_RULE) return fail(STB_ERR_INVALID_ARG, "quad_regular too large for the mixed path");
    const double pi = 3.14159265358979323846;
    dim3 grid((E + NU_THREADS - 1) / NU_THREADS, E);
    count_launch(s);
    k_regular_nu_mixed<<<grid, NU_THREADS, 0, s>>>(geo, m.d_tris, E, mrule, nq, d_cf, n_cf,
                                                   reinterpret_cast<const float4 *>(d_nodes), n_nodes,
                                                   d_targets, (float)(1.0 / (4.0 * pi * p.alpha)), V, K);
    return check_launch("k_regular_nu_mixed");
}

}  // namespace stb
