// stb_assemble_mixed.cu -- mixed-precision assembly of V^d and K^d: every
// quadrature point in FP32, no FP64 arithmetic in the hot loops.
//
// The FP64 path differences the closed-form antiderivatives (eq. vd), which
// cancels: V^d is about h^2 G while the three terms are about G^{dtau dt},
// and for far pairs at small d the true value is exponentially small.  In
// FP32 that loses every digit, so this path evaluates the same integrals in
// cancellation-free forms:
//  * d = 0, 1 from the closed forms with the part that is linear in delta
//    (exactly annihilated by the second difference) removed analytically:
//      V^0 = H(h),  V^1 = H(2h) - 2 H(h),
//      H(delta) = sqrt(delta)/(4 pi alpha^{3/2}) [ (x + 1/(2x)) erfc(x) - exp(-x^2)/sqrt(pi) ],
//    written for x(2h) < 1 with H - delta/(4 pi alpha rho) =
//      sqrt(delta)/(4 pi alpha^{3/2}) [ x erfc(x) - erf(x)/(2x) - exp(-x^2)/sqrt(pi) ],
//    and K^0, K^1 from eq. K0 / eq. K_d in the same way (see k_d01);
//  * d >= 2 from the definition eq. V_d reduced to one time variable,
//      V^d(r) = int_{-h}^{h} (h - |s|) G(r, dh + s) ds,   K^d: G -> (r.n_y)/(2 delta) G,
//    by Gauss-Legendre on every interval [kh, (k+1)h] (6 nodes for k = 1,
//    then 4, 3 or 2 as k grows, see mixed_chunk_ng); one exp2 per node feeds
//    two blocks (d = k, k + 1).
// The regularised rules of touching pairs are stored in difference form so
// that x - y keeps its relative accuracy as it shrinks.
#include <climits>
#include <cmath>
#include <vector>

#include "stb_assemble.h"
#include "stb_mixed_math.h"

namespace stb {

struct MixConsts {
    float c1, c2;    // 1/(2 sqrt(alpha h)), 1/(2 sqrt(2 alpha h))
    float ic1, ic2;  // 1/c1, 1/c2
    float pV1, pV2;  // sqrt(h)/(4 pi alpha^{3/2}), sqrt(2h)/(4 pi alpha^{3/2})
    float pK;        // 1/(4 pi alpha)
};

// Blocks d = 0 and d = 1 of one quadrature point, without the factor of the
// quadrature weight: V^0, V^1 and K^0 / (r.n), K^1 / (r.n).
__device__ __forceinline__ void k_d01(float rho, float irho, const MixConsts &g, float &v0,
                                      float &v1, float &k0, float &k1) {
    const float x1 = rho * g.c1, x2 = rho * g.c2;
    const float ix1 = irho * g.ic1, ix2 = irho * g.ic2;
    const float ec1 = erfcf(x1), ec2 = erfcf(x2);
    const float ee1 = expf(-x1 * x1), ee2 = expf(-x2 * x2);
    const float H1 = g.pV1 * ((x1 + 0.5f * ix1) * ec1 - ee1 * ISQRTPI);
    v0 = H1;
    const float kf = g.pK * irho;  // K = r.n / (4 pi alpha rho) * bracket
    k0 = kf * (ec1 * (0.25f * ix1 * ix1 - 0.5f) + 0.5f * ISQRTPI * ee1 * ix1);
    if (x2 < 1.0f) {
        const float ef1 = erff(x1), ef2 = erff(x2);
        const float Hh1 = g.pV1 * (x1 * ec1 - 0.5f * ef1 * ix1 - ee1 * ISQRTPI);
        const float Hh2 = g.pV2 * (x2 * ec2 - 0.5f * ef2 * ix2 - ee2 * ISQRTPI);
        v1 = Hh2 - 2.0f * Hh1;
        k1 = -kf * (2.0f * psi32(x1, ix1, ef1, ee1) - psi32(x2, ix2, ef2, ee2) - 0.5f);
    } else {
        const float H2 = g.pV2 * ((x2 + 0.5f * ix2) * ec2 - ee2 * ISQRTPI);
        v1 = H2 - 2.0f * H1;
        // 1/2 - psi(x) minus its part linear in delta: erfc(x)(1/2 - 1/(4x^2)) - exp(-x^2)/(2 sqrt(pi) x)
        const float c1h = ec1 * (0.5f - 0.25f * ix1 * ix1) - 0.5f * ISQRTPI * ee1 * ix1;
        const float c2h = ec2 * (0.5f - 0.25f * ix2 * ix2) - 0.5f * ISQRTPI * ee2 * ix2;
        k1 = -kf * (-2.0f * c1h + c2h);
    }
}

// Node sums of one interval k >= 2 (NG nodes, table `iv`, see stb_assemble.h)
// for NP points with squared distances rr2[p] = (rr, rr): fall[p] =
// (sum cVf e, sum cKf e) feeds block k, rise[p] = (sum cVr e, sum cKr e)
// feeds block k + 1, e = exp2(rr b).  The table entries are loaded once for
// all NP points.
template <int NG, int NP, bool SMEM>
__device__ __forceinline__ void interval_sums(const float *iv, const float2 (&rr2)[NP],
                                              float2 (&fall)[NP], float2 (&rise)[NP]) {
    const float4 b = ld_tab<SMEM>(iv);
    float e[NP][4];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const float2 t01 = __fmul2_rn(rr2[p], make_float2(b.x, b.y));
        e[p][0] = ex2(t01.x);
        e[p][1] = ex2(t01.y);
        if (NG == 3) {
            e[p][2] = ex2(rr2[p].x * b.z);
        } else if (NG == 4) {
            const float2 t23 = __fmul2_rn(rr2[p], make_float2(b.z, b.w));
            e[p][2] = ex2(t23.x);
            e[p][3] = ex2(t23.y);
        }
        fall[p] = make_float2(0.f, 0.f);
        rise[p] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < NG; ++q) {
        const float4 c = ld_tab<SMEM>(iv + 4 + 4 * q);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const float2 ee = make_float2(e[p][q], e[p][q]);
            fall[p] = __ffma2_rn(make_float2(c.x, c.y), ee, fall[p]);
            rise[p] = __ffma2_rn(make_float2(c.z, c.w), ee, rise[p]);
        }
    }
}

template <class T> __device__ __forceinline__ void store_m(T *p, float v);
template <> __device__ __forceinline__ void store_m<double>(double *p, float v) { *p = (double)v; }
template <> __device__ __forceinline__ void store_m<float>(float *p, float v) { *p = v; }

constexpr int MREG_THREADS = 128;
constexpr int MAX_RULE_M = 256;

// Intervals per pass over the quadrature points of a pair.
constexpr int MIX_G = 8;

// Node sums of MIX_G intervals (tables at tab, stride 4 + 4 NG floats) for one
// quadrature point: E[g][.] += w e, F[g][.] += w (r.n_y) e, e = exp2(rr b), with
// the nodes packed in pairs ((0,1), (2,3)) so that one packed FMA serves two.
template <int NG>
__device__ __forceinline__ void point_nodes(const float *tab, float2 rr2, float2 w2, float2 wrn2,
                                            float2 (&E)[MIX_G][2], float2 (&F)[MIX_G][2]) {
#pragma unroll
    for (int g = 0; g < MIX_G; ++g) {
        const float4 b = ld_tab<true>(tab + g * (4 + 4 * NG));
        const float2 t01 = __fmul2_rn(rr2, make_float2(b.x, b.y));
        const float2 e01 = make_float2(ex2(t01.x), ex2(t01.y));
        E[g][0] = __ffma2_rn(w2, e01, E[g][0]);
        F[g][0] = __ffma2_rn(wrn2, e01, F[g][0]);
        if (NG == 4) {
            const float2 t23 = __fmul2_rn(rr2, make_float2(b.z, b.w));
            const float2 e23 = make_float2(ex2(t23.x), ex2(t23.y));
            E[g][1] = __ffma2_rn(w2, e23, E[g][1]);
            F[g][1] = __ffma2_rn(wrn2, e23, F[g][1]);
        } else if (NG == 3) {
            const float e2 = ex2(rr2.x * b.z);
            E[g][1].x = fmaf(w2.x, e2, E[g][1].x);
            F[g][1].x = fmaf(wrn2.x, e2, F[g][1].x);
        }
    }
}

// Chunk of blocks d0..d0+MIX_CH-1 of one separated pair: the intervals
// k = d0..d0+MIX_CH-1 in passes of MIX_G over all nq x nq points.  Per pass
// the points are contracted first (E, F: sums of w e and w (r.n_y) e per
// interval and node), then the node weights are applied once per interval:
// falling side -> acc[u] (block k = d0 + u), rising side -> acc[u + 1].
// n_pass: passes holding at least one interval k <= n_steps - 1.
template <int NG>
__device__ __forceinline__ void chunk_sum(const float *tab, int n_pass,
                                          const float *__restrict__ rule, int nq,
                                          const float4 *xa, const float (&D)[3],
                                          const float (&B1)[3], const float (&B2)[3],
                                          const float (&n)[3], float2 (&acc)[MIX_CH + 1]) {
    constexpr int IVF = 4 + 4 * NG;
#pragma unroll
    for (int pass = 0; pass < MIX_CH / MIX_G; ++pass) {
        if (pass >= n_pass) break;
        const float *tg = tab + pass * MIX_G * IVF;
        float2 E[MIX_G][2], F[MIX_G][2];
#pragma unroll
        for (int g = 0; g < MIX_G; ++g)
            E[g][0] = E[g][1] = F[g][0] = F[g][1] = make_float2(0.f, 0.f);
        for (int b = 0; b < nq; ++b) {
            const float t1 = rule[4 * b], t2 = rule[4 * b + 1], wb = rule[4 * b + 2];
            const float r0b = D[0] - (t1 * B1[0] + t2 * B2[0]);
            const float r1b = D[1] - (t1 * B1[1] + t2 * B2[1]);
            const float r2b = D[2] - (t1 * B1[2] + t2 * B2[2]);
            for (int a = 0; a < nq; ++a) {
                const float4 xq = xa[a];
                const float r0 = r0b + xq.x, r1 = r1b + xq.y, r2 = r2b + xq.z;
                const float rr = r0 * r0 + r1 * r1 + r2 * r2;
                const float rn = r0 * n[0] + r1 * n[1] + r2 * n[2];
                const float w = xq.w * wb, wrn = w * rn;
                point_nodes<NG>(tg, make_float2(rr, rr), make_float2(w, w), make_float2(wrn, wrn),
                                E, F);
            }
        }
#pragma unroll
        for (int g = 0; g < MIX_G; ++g) {
            const float *iv = tg + g * IVF;
            const float Eq[4] = {E[g][0].x, E[g][0].y, E[g][1].x, E[g][1].y};
            const float Fq[4] = {F[g][0].x, F[g][0].y, F[g][1].x, F[g][1].y};
            float2 fall = make_float2(0.f, 0.f), rise = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < NG; ++q) {
                const float4 c = ld_tab<true>(iv + 4 + 4 * q);
                fall = __ffma2_rn(make_float2(c.x, c.y), make_float2(Eq[q], Fq[q]), fall);
                rise = __ffma2_rn(make_float2(c.z, c.w), make_float2(Eq[q], Fq[q]), rise);
            }
            const int u = pass * MIX_G + g;
            acc[u] = __fadd2_rn(acc[u], fall);
            acc[u + 1] = __fadd2_rn(acc[u + 1], rise);
        }
    }
}

// Test points of row l into shared memory: x_a - P0_l (FP32) and w_a.
__device__ __forceinline__ void load_test_points(const double *__restrict__ gl,
                                                 const float *__restrict__ rule, int nq,
                                                 float4 *xa) {
    for (int a = threadIdx.x; a < nq; a += blockDim.x) {
        double s1 = rule[4 * a], s2 = rule[4 * a + 1];
        double p[3];
        for (int c = 0; c < 3; ++c)
            p[c] = s1 * (gl[GEO_V1 + c] - gl[GEO_V0 + c]) + s2 * (gl[GEO_V2 + c] - gl[GEO_V1 + c]);
        xa[a] = make_float4((float)p[0], (float)p[1], (float)p[2], rule[4 * a + 2]);
    }
}

// All blocks of V (and K, unless null) for the ordered pair (l, j) of one
// problem; touching pairs are left to the regularised-rule kernel.  xa: the
// test points of row l, nd: the time-node table (both in shared memory).
template <class OutT>
__device__ __forceinline__ void regular_pair_mixed(const double *__restrict__ geo,
                                                   const int32_t *__restrict__ tris, int E,
                                                   const float *__restrict__ rule, int nq,
                                                   const float4 *xa, const float *nd,
                                                   int n_steps, const MixConsts &g,
                                                   OutT *__restrict__ V, OutT *__restrict__ K,
                                                   int l, int j) {
    const int32_t tl[3] = {tris[3 * l], tris[3 * l + 1], tris[3 * l + 2]};
    const int32_t tj[3] = {tris[3 * j], tris[3 * j + 1], tris[3 * j + 2]};
    {
        bool t = false;
        for (int i = 0; i < 3; ++i) t |= (tl[i] == tj[0]) | (tl[i] == tj[1]) | (tl[i] == tj[2]);
        if (t) return;
    }
    const double *gl = geo + (size_t)l * GEO_STRIDE, *gj = geo + (size_t)j * GEO_STRIDE;
    float D[3], B1[3], B2[3], n[3];
    for (int c = 0; c < 3; ++c) {
        D[c] = (float)(gl[GEO_V0 + c] - gj[GEO_V0 + c]);
        B1[c] = (float)(gj[GEO_V1 + c] - gj[GEO_V0 + c]);
        B2[c] = (float)(gj[GEO_V2 + c] - gj[GEO_V1 + c]);
        n[c] = (float)gj[GEO_N + c];
    }
    const float scale = (float)(4.0 * gl[GEO_AREA] * gj[GEO_AREA]);
    const size_t EE = (size_t)E * E, ij = (size_t)l * E + j;

    // pass 1: blocks 0 and 1 (closed forms) and the k = 1 interval of block 2
    float v0 = 0.f, v1 = 0.f, k0 = 0.f, k1 = 0.f, v2 = 0.f, k2 = 0.f;
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
            const float rn = r0 * n[0] + r1 * n[1] + r2 * n[2];
            const float w = xq.w * wb, wrn = w * rn;
            float a0, a1, c0, c1;
            k_d01(rho, irho, g, a0, a1, c0, c1);
            v0 = fmaf(w, a0, v0);
            v1 = fmaf(w, a1, v1);
            k0 = fmaf(wrn, c0, k0);
            k1 = fmaf(wrn, c1, k1);
            if (n_steps > 2) {
#pragma unroll
                for (int q = 0; q < MIX_NG1; ++q) {
                    const float4 c = reinterpret_cast<const float4 *>(nd)[q];
                    const float e = ex2(rr * c.x);
                    v2 = fmaf(w * c.y, e, v2);
                    k2 = fmaf(wrn * c.z, e, k2);
                }
            }
        }
    }
    store_m(V + ij, scale * v0);
    if (K) store_m(K + ij, scale * k0);
    if (n_steps > 1) {
        store_m(V + EE + ij, scale * v1);
        if (K) store_m(K + EE + ij, scale * k1);
    }

    // blocks d >= 2 in chunks of MIX_CH; chunk d0 evaluates the intervals
    // k = d0..d0+MIX_CH-1, and the rising side of interval d0-1 (from the
    // previous chunk, or pass 1 for d0 = 2) is carried into block d0
    const float *tab = nd + MIX_K1;
    float2 carry = make_float2(v2, k2);
    for (int d0 = 2; d0 < n_steps; d0 += MIX_CH) {
        float2 acc[MIX_CH + 1];
        acc[0] = carry;
#pragma unroll
        for (int u = 1; u <= MIX_CH; ++u) acc[u] = make_float2(0.f, 0.f);
        const int ng = mixed_chunk_ng(d0);
        const int n_pass = (min(MIX_CH, n_steps - d0) + MIX_G - 1) / MIX_G;
        if (ng == 4)
            chunk_sum<4>(tab, n_pass, rule, nq, xa, D, B1, B2, n, acc);
        else if (ng == 3)
            chunk_sum<3>(tab, n_pass, rule, nq, xa, D, B1, B2, n, acc);
        else
            chunk_sum<2>(tab, n_pass, rule, nq, xa, D, B1, B2, n, acc);
#pragma unroll
        for (int u = 0; u < MIX_CH; ++u) {
            const int d = d0 + u;
            if (d < n_steps) {
                store_m(V + (size_t)d * EE + ij, scale * acc[u].x);
                if (K) store_m(K + (size_t)d * EE + ij, scale * acc[u].y);
            }
        }
        carry = acc[MIX_CH];
        tab += MIX_CH * mixed_iv_floats(ng);
    }
}


template <class OutT>
__global__ void __launch_bounds__(MREG_THREADS)
k_regular_mixed(const double *__restrict__ geo, const int32_t *__restrict__ tris, int E,
                const float *__restrict__ rule, int nq, const float *__restrict__ nodes,
                int n_nodes_f, int n_steps, MixConsts g, OutT *__restrict__ V,
                OutT *__restrict__ K) {
    extern __shared__ float smf[];
    float4 *xa = reinterpret_cast<float4 *>(smf);  // x_a - P0_l and w_a
    float *nd = smf + 4 * MAX_RULE_M;             // time nodes
    const int l = blockIdx.y;
    const int j = blockIdx.x * MREG_THREADS + threadIdx.x;
    load_test_points(geo + (size_t)l * GEO_STRIDE, rule, nq, xa);
    for (int i = threadIdx.x; i < n_nodes_f; i += MREG_THREADS) nd[i] = nodes[i];
    __syncthreads();
    if (j < E) regular_pair_mixed<OutT>(geo, tris, E, rule, nq, xa, nd, n_steps, g, V, K, l, j);
}

// ------------------------------------------------------- touching pairs ---
constexpr int MSS_THREADS = 128;

// One chunk of a touching pair's blocks for one point: intervals
// k = d0 + u (u < CH); the falling side feeds block k (index u), the rising
// side block k + 1 (index u + 1, u + 1 = CH being the carry into the next
// chunk): acc[i] (V), acc[CH + 1 + i] (K at (a,b)), acc[2 (CH + 1) + i] (K at (b,a)).
template <int NG, int CH>
__device__ __forceinline__ void ss_chunk(const float *tab, int d0, int n_steps, float rr, float w,
                                         float wa, float wb, float (&acc)[3 * (CH + 1)]) {
    const float2 rr2[1] = {make_float2(rr, rr)};
    constexpr int S = CH + 1;
#pragma unroll
    for (int u = 0; u < CH; ++u) {
        if (d0 + u > n_steps - 1) break;
        float2 fall[1], rise[1];
        interval_sums<NG, 1, false>(tab + u * (4 + 4 * NG), rr2, fall, rise);
        acc[u] = fmaf(w, fall[0].x, acc[u]);
        acc[S + u] = fmaf(wa, fall[0].y, acc[S + u]);
        acc[2 * S + u] = fmaf(wb, fall[0].y, acc[2 * S + u]);
        acc[u + 1] = fmaf(w, rise[0].x, acc[u + 1]);
        acc[S + u + 1] = fmaf(wa, rise[0].y, acc[S + u + 1]);
        acc[2 * S + u + 1] = fmaf(wb, rise[0].y, acc[2 * S + u + 1]);
    }
}

struct MixSS {
    const float *p0[4], *p1[4], *p2[4], *p3[4], *w[4];
    int n[4];
};

// All blocks of the touching pair P (both orders) of one problem: the first
// NTH threads of the CTA (at least 3 CH + 9) share the points of the
// regularised rule; further threads of a larger CTA take part only in its
// barriers, so the sums (and their rounding) do not depend on the CTA size.
// kp (optional): instead of K, the pair's K blocks go to kp[d] (entry (a,b))
// and kp[n_steps + d] (entry (b,a)).
template <int CH, class OutT, int NTH = MSS_THREADS>
__device__ __forceinline__ void singular_pair_mixed(const double *__restrict__ geo,
                                                    const TouchPair P, int E, const MixSS &tab,
                                                    const float *__restrict__ nodes, int n_steps,
                                                    const MixConsts &g, OutT *__restrict__ V,
                                                    OutT *__restrict__ K, float *kp = nullptr) {
    static_assert(NTH % 32 == 0 && NTH >= 3 * CH + 9, "one thread per reduced value");
    __shared__ float red[NTH / 32][3 * CH + 9];
    const int p_first = threadIdx.x < NTH ? (int)threadIdx.x : INT_MAX;  // first rule point
    __shared__ float fin[3 * CH + 9];
    const int a = P.a, b = P.b, cls = P.cls;
    if (a < 0 || b < a || b >= E || cls < PAIR_VERTEX || cls > PAIR_IDENTICAL) return;
    const double *ga = geo + (size_t)a * GEO_STRIDE, *gb = geo + (size_t)b * GEO_STRIDE;
    // x - y = p0 X0 + p1 X1 + p2 X2 + p3 X3 (difference form of the rule)
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
    const float scale = (float)(4.0 * ga[GEO_AREA] * gb[GEO_AREA]);
    const bool ident = cls == PAIR_IDENTICAL;
    const int npt = tab.n[cls];
    const float *R0 = tab.p0[cls], *R1 = tab.p1[cls], *R2 = tab.p2[cls], *R3 = tab.p3[cls],
                *W = tab.w[cls];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t EE = (size_t)E * E, iab = (size_t)a * E + b, iba = (size_t)b * E + a;

    // entry (a,b): r = x - y, n_b; entry (b,a): r' = -r, n_a
    auto point = [&](int p, float &rr, float &rab, float &rba, float &w) {
        const float q0 = R0[p], q1 = R1[p], q2 = R2[p], q3 = R3[p];
        float r[3];
        for (int c = 0; c < 3; ++c) r[c] = q0 * X[0][c] + q1 * X[1][c] + q2 * X[2][c] + q3 * X[3][c];
        rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        rab = r[0] * nb[0] + r[1] * nb[1] + r[2] * nb[2];
        rba = -(r[0] * na[0] + r[1] * na[1] + r[2] * na[2]);
        w = W[p];
    };
    auto reduce = [&](float *vals, int nv) {
        for (int k = 0; k < nv; ++k) {
            float v = vals[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && warp < NTH / 32) red[warp][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < nv) {
            float s = 0.f;
            for (int wi = 0; wi < NTH / 32; ++wi) s += red[wi][threadIdx.x];
            fin[threadIdx.x] = scale * s;
        }
        __syncthreads();
    };

    // pass 1: blocks 0, 1 and the k = 1 interval of block 2
    float z[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) z[i] = 0.f;
    for (int p = p_first; p < npt; p += NTH) {
        float rr, rab, rba, w;
        point(p, rr, rab, rba, w);
        const float irho = rsqrtf(rr), rho = rr * irho;
        float a0, a1, c0, c1;
        k_d01(rho, irho, g, a0, a1, c0, c1);
        z[0] = fmaf(w, a0, z[0]);
        z[1] = fmaf(w, a1, z[1]);
        z[2] = fmaf(w * rab, c0, z[2]);
        z[3] = fmaf(w * rab, c1, z[3]);
        z[4] = fmaf(w * rba, c0, z[4]);
        z[5] = fmaf(w * rba, c1, z[5]);
        if (n_steps > 2) {
#pragma unroll
            for (int q = 0; q < MIX_NG1; ++q) {
                const float4 c = reinterpret_cast<const float4 *>(nodes)[q];
                const float e = ex2(rr * c.x);
                z[6] = fmaf(w * c.y, e, z[6]);
                z[7] = fmaf(w * rab * c.z, e, z[7]);
                z[8] = fmaf(w * rba * c.z, e, z[8]);
            }
        }
    }
    reduce(z, 9);
    if (threadIdx.x == 0) {
        store_m(V + iab, fin[0]);
        if (!ident) store_m(V + iba, fin[0]);
        if (kp) {
            kp[0] = ident ? 0.f : fin[2];
            kp[n_steps] = ident ? 0.f : fin[4];
        } else if (K) {
            store_m(K + iab, ident ? 0.f : fin[2]);
            if (!ident) store_m(K + iba, fin[4]);
        }
        if (n_steps > 1) {
            store_m(V + EE + iab, fin[1]);
            if (!ident) store_m(V + EE + iba, fin[1]);
            if (kp) {
                kp[1] = ident ? 0.f : fin[3];
                kp[n_steps + 1] = ident ? 0.f : fin[5];
            } else if (K) {
                store_m(K + EE + iab, ident ? 0.f : fin[3]);
                if (!ident) store_m(K + EE + iba, fin[5]);
            }
        }
    }
    float cv = fin[6], ca = fin[7], cb = fin[8];  // carry into block d0 (already scaled)
    __syncthreads();

    constexpr int S = CH + 1;
    const float *ntab = nodes + MIX_K1;
    for (int d0 = 2; d0 < n_steps; d0 += CH) {
        float acc[3 * S];
#pragma unroll
        for (int i = 0; i < 3 * S; ++i) acc[i] = 0.f;
        const int ng = mixed_chunk_ng(d0);
        for (int p = p_first; p < npt; p += NTH) {
            float rr, rab, rba, w;
            point(p, rr, rab, rba, w);
            if (ng == 4) ss_chunk<4, CH>(ntab, d0, n_steps, rr, w, w * rab, w * rba, acc);
            else if (ng == 3) ss_chunk<3, CH>(ntab, d0, n_steps, rr, w, w * rab, w * rba, acc);
            else ss_chunk<2, CH>(ntab, d0, n_steps, rr, w, w * rab, w * rba, acc);
        }
        ntab += CH * mixed_iv_floats(ng);
        reduce(acc, 3 * S);
        if (threadIdx.x == 0) {
            for (int u = 0; u < CH; ++u) {
                const int d = d0 + u;
                if (d >= n_steps) break;
                float bv = fin[u], ba = fin[S + u], bb = fin[2 * S + u];
                if (u == 0) {
                    bv += cv;
                    ba += ca;
                    bb += cb;
                }
                const size_t off = (size_t)d * EE;
                store_m(V + off + iab, bv);
                if (!ident) store_m(V + off + iba, bv);
                if (kp) {
                    kp[d] = ident ? 0.f : ba;
                    kp[n_steps + d] = ident ? 0.f : bb;
                } else if (K) {
                    store_m(K + off + iab, ident ? 0.f : ba);
                    if (!ident) store_m(K + off + iba, bb);
                }
            }
        }
        cv = fin[CH];
        ca = fin[S + CH];
        cb = fin[2 * S + CH];
        __syncthreads();
    }
}

template <int CH, class OutT>
__global__ void __launch_bounds__(MSS_THREADS)
k_singular_mixed(const double *__restrict__ geo, const TouchPair *__restrict__ pairs, int E,
                 MixSS tab, const float *__restrict__ nodes, int n_steps, MixConsts g,
                 OutT *__restrict__ V, OutT *__restrict__ K) {
    singular_pair_mixed<CH, OutT>(geo, pairs[blockIdx.x], E, tab, nodes, n_steps, g, V, K);
}

// ------------------------------------------------------------ host side ---
void mixed_tables(const stb_params &p, std::vector<float> &rule, std::vector<float> &ss,
                  std::vector<float> &nodes) {
    const double pi = 3.14159265358979323846, al = p.alpha, h = p.T / p.n_steps;
    std::vector<double> a, b, c, d, w;
    triangle_rule(p.quad_regular, a, b, w);
    rule.clear();
    for (size_t i = 0; i < w.size(); ++i) {
        rule.push_back((float)a[i]);
        rule.push_back((float)b[i]);
        rule.push_back((float)w[i]);
        rule.push_back(0.f);
    }
    ss.clear();
    for (int cls = 1; cls <= 3; ++cls) {
        ss_rule_diff(cls, p.quad_singular, a, b, c, d, w);
        for (auto *v : {&a, &b, &c, &d, &w})
            for (double x : *v) ss.push_back((float)x);
    }
    nodes.assign(mixed_node_floats(p.n_steps), 0.f);
    // b = exp2 scale, wf / wr = falling / rising weights of block k / k+1
    auto node = [&](int k, double ug, double wg, double &b, double &wf, double &wr, double &delta) {
        delta = (k + ug) * h;
        const double a_ = std::pow(4.0 * pi * al * delta, -1.5);
        b = -1.0 / (4.0 * al * delta) * 1.4426950408889634;  // log2(e)
        wf = h * wg * h * (1.0 - ug) * a_;
        wr = h * wg * h * ug * a_;
    };
    std::vector<double> u1(MIX_NG1), w1(MIX_NG1), u(4), wq(4);
    gauss_legendre01(MIX_NG1, u1.data(), w1.data());
    for (int q = 0; q < MIX_NG1; ++q) {
        double b, wf, wr, delta;
        node(1, u1[q], w1[q], b, wf, wr, delta);
        float *o = nodes.data() + 4 * q;
        o[0] = (float)b;
        o[1] = (float)wr;
        o[2] = (float)(wr / (2.0 * delta));
    }
    size_t off = MIX_K1;
    for (int d0 = 2; d0 < p.n_steps; d0 += MIX_CH) {
        const int ng = mixed_chunk_ng(d0);
        gauss_legendre01(ng, u.data(), wq.data());
        for (int uu = 0; uu < MIX_CH; ++uu, off += mixed_iv_floats(ng)) {
            const int k = d0 + uu;
            if (k > p.n_steps - 1) continue;  // zero weights
            float *o = nodes.data() + off;
            for (int q = 0; q < ng; ++q) {
                double b, wf, wr, delta;
                node(k, u[q], wq[q], b, wf, wr, delta);
                o[q] = (float)b;
                o[4 + 4 * q + 0] = (float)wf;
                o[4 + 4 * q + 1] = (float)(wf / (2.0 * delta));
                o[4 + 4 * q + 2] = (float)wr;
                o[4 + 4 * q + 3] = (float)(wr / (2.0 * delta));
            }
        }
    }
}

static MixConsts mix_consts(const stb_params &p) {
    const double pi = 3.14159265358979323846, al = p.alpha, h = p.T / p.n_steps;
    MixConsts g;
    g.c1 = (float)(1.0 / (2.0 * std::sqrt(al * h)));
    g.c2 = (float)(1.0 / (2.0 * std::sqrt(2.0 * al * h)));
    g.ic1 = (float)(2.0 * std::sqrt(al * h));
    g.ic2 = (float)(2.0 * std::sqrt(2.0 * al * h));
    g.pV1 = (float)(std::sqrt(h) / (4.0 * pi * std::pow(al, 1.5)));
    g.pV2 = (float)(std::sqrt(2.0 * h) / (4.0 * pi * std::pow(al, 1.5)));
    g.pK = (float)(1.0 / (4.0 * pi * al));
    return g;
}

static MixSS mix_ss(const AssemblyLayout &L) {
    MixSS tab{};
    const float *base = L.mss;
    for (int cls = 1; cls <= 3; ++cls) {
        const size_t n = L.ss_n[cls];
        tab.p0[cls] = base;
        tab.p1[cls] = base + n;
        tab.p2[cls] = base + 2 * n;
        tab.p3[cls] = base + 3 * n;
        tab.w[cls] = base + 4 * n;
        tab.n[cls] = (int)n;
        base += 5 * n;
    }
    return tab;
}

template <class OutT>
static stb_status run_mixed_t(const Mesh &m, const stb_params &p, OutT *V, OutT *K,
                              const AssemblyLayout &L, cudaStream_t s) {
    constexpr int CH = MIX_CH;
    const int E = (int)m.n_tris;
    const int nq = p.quad_regular * p.quad_regular;
    const MixConsts g = mix_consts(p);
    const int nf = (int)mixed_node_floats(p.n_steps);
    const size_t smem = sizeof(float) * (4 * MAX_RULE_M + (size_t)nf);
    STB_CUDA(cudaFuncSetAttribute(k_regular_mixed<OutT>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((E + MREG_THREADS - 1) / MREG_THREADS, E);
    count_launch(s);
    k_regular_mixed<OutT><<<grid, MREG_THREADS, smem, s>>>(L.geo, m.d_tris, E, L.mrule, nq,
                                                               L.mnodes, nf, p.n_steps, g, V, K);
    stb_status st = check_launch("k_regular_mixed");
    if (st) return st;
    if (m.n_touch > 0) {
        const MixSS tab = mix_ss(L);
        count_launch(s);
        k_singular_mixed<CH, OutT><<<(unsigned)m.n_touch, MSS_THREADS, 0, s>>>(
            L.geo, L.pairs, E, tab, L.mnodes, p.n_steps, g, V, K);
        if ((st = check_launch("k_singular_mixed"))) return st;
    }
    return STB_OK;
}

stb_status run_assembly_mixed(const Mesh &m, const stb_params &p, void *V, void *K,
                              const AssemblyLayout &L, cudaStream_t s) {
    if (p.storage == STB_STORE_F64)
        return run_mixed_t<double>(m, p, (double *)V, (double *)K, L, s);
    return run_mixed_t<float>(m, p, (float *)V, (float *)K, L, s);
}

// ------------------------------ piecewise-linear trial space, mixed ---
// K_h with nodal hat trial functions (Sec. 3.2) in the forms of the mixed
// path: the K integrand of a pair weighted by the barycentric coordinates
// lambda_v of the trial point, added per vertex to K1[d][l][node] with FP32
// atomics (K1 starts at zero).  Separated pairs: the trial weight and
// lambda depend only on the trial point b, so the test points a are summed
// first (one packed FMA per exp2, as for the p0 blocks) and the three
// vertex weights are applied once per trial point.
constexpr int K1_G = 4;  // intervals per pass over the points

// F[g][.] += wrn e for K1_G intervals, e = exp2(rr b), nodes packed in pairs
template <int NG>
__device__ __forceinline__ void point_nodes_k1(const float *tab, float2 rr2, float2 wrn2,
                                               float2 (&F)[K1_G][2]) {
#pragma unroll
    for (int g = 0; g < K1_G; ++g) {
        const float4 b = ld_tab<true>(tab + g * (4 + 4 * NG));
        const float2 t01 = __fmul2_rn(rr2, make_float2(b.x, b.y));
        F[g][0] = __ffma2_rn(wrn2, make_float2(ex2(t01.x), ex2(t01.y)), F[g][0]);
        if (NG == 4) {
            const float2 t23 = __fmul2_rn(rr2, make_float2(b.z, b.w));
            F[g][1] = __ffma2_rn(wrn2, make_float2(ex2(t23.x), ex2(t23.y)), F[g][1]);
        } else if (NG == 3) {
            F[g][1].x = fmaf(wrn2.x, ex2(rr2.x * b.z), F[g][1].x);
        }
    }
}

// Blocks d0..d0+n_int-1 of one separated pair (the intervals k = d0.. of one
// table chunk, n_int <= MIX_CH), in passes of K1_G intervals; carry[v]: the
// rising side of interval d0-1 per vertex (scaled), updated to that of the
// last interval.  Completed blocks go out with atomics.
template <int NG>
__device__ __forceinline__ void chunk_k1(const float *tab, int d0, int n_int,
                                         const float *__restrict__ rule, int nq,
                                         const float4 *xa, const float (&D)[3],
                                         const float (&B1)[3], const float (&B2)[3],
                                         const float (&n)[3], float scale, float (&carry)[3],
                                         float *__restrict__ out, size_t EN, const int (&tj)[3]) {
    constexpr int IVF = 4 + 4 * NG;
    for (int u0 = 0; u0 < n_int; u0 += K1_G) {
        const float *tg = tab + u0 * IVF;
        float2 Fv[3][K1_G][2];
#pragma unroll
        for (int v = 0; v < 3; ++v)
#pragma unroll
            for (int g = 0; g < K1_G; ++g) Fv[v][g][0] = Fv[v][g][1] = make_float2(0.f, 0.f);
        for (int b = 0; b < nq; ++b) {
            const float t1 = rule[4 * b], t2 = rule[4 * b + 1], wb = rule[4 * b + 2];
            const float r0b = D[0] - (t1 * B1[0] + t2 * B2[0]);
            const float r1b = D[1] - (t1 * B1[1] + t2 * B2[1]);
            const float r2b = D[2] - (t1 * B1[2] + t2 * B2[2]);
            float2 Fb[K1_G][2];
#pragma unroll
            for (int g = 0; g < K1_G; ++g) Fb[g][0] = Fb[g][1] = make_float2(0.f, 0.f);
            for (int a = 0; a < nq; ++a) {
                const float4 xq = xa[a];
                const float r0 = r0b + xq.x, r1 = r1b + xq.y, r2 = r2b + xq.z;
                const float rr = r0 * r0 + r1 * r1 + r2 * r2;
                const float wrn = xq.w * (r0 * n[0] + r1 * n[1] + r2 * n[2]);
                point_nodes_k1<NG>(tg, make_float2(rr, rr), make_float2(wrn, wrn), Fb);
            }
            const float lw[3] = {(1.f - t1) * wb, (t1 - t2) * wb, t2 * wb};
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const float2 l2 = make_float2(lw[v], lw[v]);
#pragma unroll
                for (int g = 0; g < K1_G; ++g) {
                    Fv[v][g][0] = __ffma2_rn(l2, Fb[g][0], Fv[v][g][0]);
                    Fv[v][g][1] = __ffma2_rn(l2, Fb[g][1], Fv[v][g][1]);
                }
            }
        }
#pragma unroll
        for (int g = 0; g < K1_G; ++g) {
            if (u0 + g >= n_int) break;
            const float *iv = tg + g * IVF;
            float fall[3] = {0.f, 0.f, 0.f}, rise[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < NG; ++q) {
                const float4 c = ld_tab<true>(iv + 4 + 4 * q);  // (cVf, cKf, cVr, cKr)
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const float f = (q & 1) ? Fv[v][g][q >> 1].y : Fv[v][g][q >> 1].x;
                    fall[v] = fmaf(c.y, f, fall[v]);
                    rise[v] = fmaf(c.w, f, rise[v]);
                }
            }
            float *blk = out + (size_t)(d0 + u0 + g) * EN;
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                atomicAdd(blk + tj[v], fmaf(scale, fall[v], carry[v]));
                carry[v] = scale * rise[v];
            }
        }
    }
}

// All blocks of K1 for the separated ordered pair (l, j).
__device__ __forceinline__ void regular_pair_k1_mixed(const double *__restrict__ geo,
                                                      const int32_t *__restrict__ tris, int E,
                                                      int N, const float *__restrict__ rule,
                                                      int nq, const float4 *xa, const float *nd,
                                                      int n_steps, const MixConsts &g,
                                                      float *__restrict__ K1, int l, int j) {
    const int32_t tl[3] = {tris[3 * l], tris[3 * l + 1], tris[3 * l + 2]};
    const int tj[3] = {tris[3 * j], tris[3 * j + 1], tris[3 * j + 2]};
    {
        bool t = false;
        for (int i = 0; i < 3; ++i) t |= (tl[i] == tj[0]) | (tl[i] == tj[1]) | (tl[i] == tj[2]);
        if (t) return;
    }
    const double *gl = geo + (size_t)l * GEO_STRIDE, *gj = geo + (size_t)j * GEO_STRIDE;
    float D[3], B1[3], B2[3], n[3];
    for (int c = 0; c < 3; ++c) {
        D[c] = (float)(gl[GEO_V0 + c] - gj[GEO_V0 + c]);
        B1[c] = (float)(gj[GEO_V1 + c] - gj[GEO_V0 + c]);
        B2[c] = (float)(gj[GEO_V2 + c] - gj[GEO_V1 + c]);
        n[c] = (float)gj[GEO_N + c];
    }
    const float scale = (float)(4.0 * gl[GEO_AREA] * gj[GEO_AREA]);
    const size_t EN = (size_t)E * N;
    float *out = K1 + (size_t)l * N;

    // pass 1: blocks 0 and 1 (closed forms) and the k = 1 interval of block 2
    float k0[3] = {0.f, 0.f, 0.f}, k1[3] = {0.f, 0.f, 0.f}, k2[3] = {0.f, 0.f, 0.f};
    for (int b = 0; b < nq; ++b) {
        const float t1 = rule[4 * b], t2 = rule[4 * b + 1], wb = rule[4 * b + 2];
        const float r0b = D[0] - (t1 * B1[0] + t2 * B2[0]);
        const float r1b = D[1] - (t1 * B1[1] + t2 * B2[1]);
        const float r2b = D[2] - (t1 * B1[2] + t2 * B2[2]);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int a = 0; a < nq; ++a) {
            const float4 xq = xa[a];
            const float r0 = r0b + xq.x, r1 = r1b + xq.y, r2 = r2b + xq.z;
            const float rr = r0 * r0 + r1 * r1 + r2 * r2;
            const float irho = rsqrtf(rr), rho = rr * irho;
            const float wrn = xq.w * (r0 * n[0] + r1 * n[1] + r2 * n[2]);
            float a0, a1, c0, c1;
            k_d01(rho, irho, g, a0, a1, c0, c1);
            s0 = fmaf(wrn, c0, s0);
            s1 = fmaf(wrn, c1, s1);
            if (n_steps > 2) {
#pragma unroll
                for (int q = 0; q < MIX_NG1; ++q) {
                    const float4 c = reinterpret_cast<const float4 *>(nd)[q];
                    s2 = fmaf(wrn * c.z, ex2(rr * c.x), s2);
                }
            }
        }
        const float lw[3] = {(1.f - t1) * wb, (t1 - t2) * wb, t2 * wb};
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            k0[v] = fmaf(lw[v], s0, k0[v]);
            k1[v] = fmaf(lw[v], s1, k1[v]);
            k2[v] = fmaf(lw[v], s2, k2[v]);
        }
    }
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        atomicAdd(out + tj[v], scale * k0[v]);
        if (n_steps > 1) atomicAdd(out + EN + tj[v], scale * k1[v]);
    }
    float carry[3] = {scale * k2[0], scale * k2[1], scale * k2[2]};
    const float *tab = nd + MIX_K1;
    for (int d0 = 2; d0 < n_steps; d0 += MIX_CH) {
        const int ng = mixed_chunk_ng(d0), n_int = min(MIX_CH, n_steps - d0);
        if (ng == 4)
            chunk_k1<4>(tab, d0, n_int, rule, nq, xa, D, B1, B2, n, scale, carry, out, EN, tj);
        else if (ng == 3)
            chunk_k1<3>(tab, d0, n_int, rule, nq, xa, D, B1, B2, n, scale, carry, out, EN, tj);
        else
            chunk_k1<2>(tab, d0, n_int, rule, nq, xa, D, B1, B2, n, scale, carry, out, EN, tj);
        tab += MIX_CH * mixed_iv_floats(ng);
    }
}

__global__ void __launch_bounds__(MREG_THREADS)
k_regular_k1_mixed(const double *__restrict__ geo, const int32_t *__restrict__ tris, int E, int N,
                   const float *__restrict__ rule, int nq, const float *__restrict__ nodes,
                   int n_nodes_f, int n_steps, MixConsts g, float *__restrict__ K1) {
    extern __shared__ float smf[];
    float4 *xa = reinterpret_cast<float4 *>(smf);
    float *nd = smf + 4 * MAX_RULE_M;
    const int l = blockIdx.y;
    const int j = blockIdx.x * MREG_THREADS + threadIdx.x;
    load_test_points(geo + (size_t)l * GEO_STRIDE, rule, nq, xa);
    for (int i = threadIdx.x; i < n_nodes_f; i += MREG_THREADS) nd[i] = nodes[i];
    __syncthreads();
    if (j < E) regular_pair_k1_mixed(geo, tris, E, N, rule, nq, xa, nd, n_steps, g, K1, l, j);
}

// Touching pairs: one CTA per unordered pair (a, b), the difference-form
// rule for r and the rule's coordinates (s1, s2) on a, (t1, t2) on b in the
// pair's rotated vertex orders for the barycentric weights: entry (a, b) has
// its trial point on b, entry (b, a) on a.  Identical pairs give zero.
// Sub-chunks of K1_SCH intervals keep 6 (K1_SCH + 1) sums per thread.
constexpr int K1_SCH = 8;

struct MixK1Coords {
    const float *s1[4], *s2[4], *t1[4], *t2[4];
};

__global__ void __launch_bounds__(MSS_THREADS)
k_singular_k1_mixed(const double *__restrict__ geo, const int32_t *__restrict__ tris,
                    const TouchPair *__restrict__ pairs, int E, int N, MixSS tab, MixK1Coords co,
                    const float *__restrict__ nodes, int n_steps, MixConsts g,
                    float *__restrict__ K1) {
    constexpr int S = K1_SCH + 1;
    __shared__ float red[MSS_THREADS / 32][6 * S];
    __shared__ float fin[6 * S];
    const TouchPair P = pairs[blockIdx.x];
    const int a = P.a, b = P.b, cls = P.cls;
    if (a < 0 || b < a || b >= E || cls < PAIR_VERTEX || cls >= PAIR_IDENTICAL) return;
    const double *ga = geo + (size_t)a * GEO_STRIDE, *gb = geo + (size_t)b * GEO_STRIDE;
    const int oa[3] = {P.perm & 3, (P.perm >> 2) & 3, (P.perm >> 4) & 3};
    const int ob[3] = {(P.perm >> 6) & 3, (P.perm >> 8) & 3, (P.perm >> 10) & 3};
    float X[4][3], na[3], nb[3];
    for (int c = 0; c < 3; ++c) {
        const double A1 = ga[3 * oa[1] + c] - ga[3 * oa[0] + c], A2 = ga[3 * oa[2] + c] - ga[3 * oa[1] + c];
        const double Bv1 = gb[3 * ob[1] + c] - gb[3 * ob[0] + c], Bv2 = gb[3 * ob[2] + c] - gb[3 * ob[1] + c];
        if (cls == PAIR_EDGE) {
            X[0][c] = (float)-A1; X[1][c] = (float)A2; X[2][c] = (float)-Bv2; X[3][c] = 0.f;
        } else {
            X[0][c] = (float)A1; X[1][c] = (float)A2; X[2][c] = (float)-Bv1; X[3][c] = (float)-Bv2;
        }
        na[c] = (float)ga[GEO_N + c];
        nb[c] = (float)gb[GEO_N + c];
    }
    int nodes_a[3], nodes_b[3];
    for (int c = 0; c < 3; ++c) {
        nodes_a[c] = tris[3 * a + oa[c]];
        nodes_b[c] = tris[3 * b + ob[c]];
    }
    const float scale = (float)(4.0 * ga[GEO_AREA] * gb[GEO_AREA]);
    const int npt = tab.n[cls];
    const float *R0 = tab.p0[cls], *R1 = tab.p1[cls], *R2 = tab.p2[cls], *R3 = tab.p3[cls],
                *W = tab.w[cls];
    const float *S1 = co.s1[cls], *S2 = co.s2[cls], *T1 = co.t1[cls], *T2 = co.t2[cls];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t EN = (size_t)E * N;

    // point p: r^2 and the weights w (r.n_b) lambda_b(t) (entry (a,b)) and
    // w (r'.n_a) lambda_a(s) (entry (b,a), r' = -r)
    auto point = [&](int p, float &rr, float (&wab)[3], float (&wba)[3]) {
        const float q0 = R0[p], q1 = R1[p], q2 = R2[p], q3 = R3[p];
        float r[3];
        for (int c = 0; c < 3; ++c) r[c] = q0 * X[0][c] + q1 * X[1][c] + q2 * X[2][c] + q3 * X[3][c];
        rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        const float w = W[p];
        const float rab = w * (r[0] * nb[0] + r[1] * nb[1] + r[2] * nb[2]);
        const float rba = -w * (r[0] * na[0] + r[1] * na[1] + r[2] * na[2]);
        const float s1 = S1[p], s2 = S2[p], t1 = T1[p], t2 = T2[p];
        wab[0] = rab * (1.f - t1); wab[1] = rab * (t1 - t2); wab[2] = rab * t2;
        wba[0] = rba * (1.f - s1); wba[1] = rba * (s1 - s2); wba[2] = rba * s2;
    };
    auto reduce = [&](float *vals, int nv) {
        for (int k = 0; k < nv; ++k) {
            float v = vals[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < nv) {
            float sum = 0.f;
            for (int wi = 0; wi < MSS_THREADS / 32; ++wi) sum += red[wi][threadIdx.x];
            fin[threadIdx.x] = scale * sum;
        }
        __syncthreads();
    };
    // entry e (0..2: (a,b) at node nodes_b[e]; 3..5: (b,a) at node nodes_a[e-3])
    auto emit = [&](int d, int e, float val) {
        float *blk = K1 + (size_t)d * EN;
        if (e < 3)
            atomicAdd(blk + (size_t)a * N + nodes_b[e], val);
        else
            atomicAdd(blk + (size_t)b * N + nodes_a[e - 3], val);
    };

    // pass 1: blocks 0, 1 and the k = 1 interval of block 2 (18 sums)
    float z[18];
#pragma unroll
    for (int i = 0; i < 18; ++i) z[i] = 0.f;
    for (int p = threadIdx.x; p < npt; p += MSS_THREADS) {
        float rr, wab[3], wba[3];
        point(p, rr, wab, wba);
        const float irho = rsqrtf(rr), rho = rr * irho;
        float a0, a1, c0, c1;
        k_d01(rho, irho, g, a0, a1, c0, c1);
        float c2 = 0.f;
        if (n_steps > 2) {
#pragma unroll
            for (int q = 0; q < MIX_NG1; ++q) {
                const float4 c = reinterpret_cast<const float4 *>(nodes)[q];
                c2 = fmaf(c.z, ex2(rr * c.x), c2);
            }
        }
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            z[v] = fmaf(wab[v], c0, z[v]);
            z[3 + v] = fmaf(wba[v], c0, z[3 + v]);
            z[6 + v] = fmaf(wab[v], c1, z[6 + v]);
            z[9 + v] = fmaf(wba[v], c1, z[9 + v]);
            z[12 + v] = fmaf(wab[v], c2, z[12 + v]);
            z[15 + v] = fmaf(wba[v], c2, z[15 + v]);
        }
    }
    reduce(z, 18);
    if (threadIdx.x == 0) {
        for (int e = 0; e < 6; ++e) {
            emit(0, e, fin[e]);
            if (n_steps > 1) emit(1, e, fin[6 + e]);
        }
    }
    float carry[6];
    for (int e = 0; e < 6; ++e) carry[e] = fin[12 + e];
    __syncthreads();

    const float *ntab = nodes + MIX_K1;
    for (int d0 = 2; d0 < n_steps; d0 += MIX_CH) {
        const int ng = mixed_chunk_ng(d0), ivf = mixed_iv_floats(ng);
        for (int h0 = 0; h0 < MIX_CH && d0 + h0 < n_steps; h0 += K1_SCH) {
            const int n_int = min(K1_SCH, n_steps - d0 - h0);
            float acc[6 * S];
#pragma unroll
            for (int i = 0; i < 6 * S; ++i) acc[i] = 0.f;
            const float *tb = ntab + h0 * ivf;
            for (int p = threadIdx.x; p < npt; p += MSS_THREADS) {
                float rr, wab[3], wba[3];
                point(p, rr, wab, wba);
                const float2 rr2[1] = {make_float2(rr, rr)};
#pragma unroll
                for (int u = 0; u < K1_SCH; ++u) {
                    if (u >= n_int) break;
                    float2 fall[1], rise[1];
                    if (ng == 4) interval_sums<4, 1, false>(tb + u * ivf, rr2, fall, rise);
                    else if (ng == 3) interval_sums<3, 1, false>(tb + u * ivf, rr2, fall, rise);
                    else interval_sums<2, 1, false>(tb + u * ivf, rr2, fall, rise);
#pragma unroll
                    for (int v = 0; v < 3; ++v) {
                        acc[v * S + u] = fmaf(wab[v], fall[0].y, acc[v * S + u]);
                        acc[v * S + u + 1] = fmaf(wab[v], rise[0].y, acc[v * S + u + 1]);
                        acc[(3 + v) * S + u] = fmaf(wba[v], fall[0].y, acc[(3 + v) * S + u]);
                        acc[(3 + v) * S + u + 1] = fmaf(wba[v], rise[0].y, acc[(3 + v) * S + u + 1]);
                    }
                }
            }
            reduce(acc, 6 * S);
            if (threadIdx.x == 0) {
                for (int u = 0; u < n_int; ++u)
                    for (int e = 0; e < 6; ++e)
                        emit(d0 + h0 + u, e, fin[e * S + u] + (u == 0 ? carry[e] : 0.f));
            }
            for (int e = 0; e < 6; ++e) carry[e] = fin[e * S + n_int];
            __syncthreads();
        }
        ntab += MIX_CH * ivf;
    }
}

stb_status run_assembly_k1_mixed(const Mesh &m, const stb_params &p, float *K1,
                                 const AssemblyLayout &L, const float *coords, cudaStream_t s) {
    const int E = (int)m.n_tris, N = (int)m.n_nodes;
    const int nq = p.quad_regular * p.quad_regular;
    const MixConsts g = mix_consts(p);
    const int nf = (int)mixed_node_floats(p.n_steps);
    STB_CUDA(cudaMemsetAsync(K1, 0, sizeof(float) * (size_t)p.n_steps * E * N, s));
    const size_t smem = sizeof(float) * (4 * MAX_RULE_M + (size_t)nf);
    STB_CUDA(cudaFuncSetAttribute(k_regular_k1_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    dim3 grid((E + MREG_THREADS - 1) / MREG_THREADS, E);
    count_launch(s);
    k_regular_k1_mixed<<<grid, MREG_THREADS, smem, s>>>(L.geo, m.d_tris, E, N, L.mrule, nq,
                                                         L.mnodes, nf, p.n_steps, g, K1);
    stb_status st = check_launch("k_regular_k1_mixed");
    if (st || m.n_touch == 0) return st;
    const MixSS tab = mix_ss(L);
    MixK1Coords co{};
    const float *base = coords;
    for (int cls = 1; cls <= 3; ++cls) {
        const size_t n = L.ss_n[cls];
        co.s1[cls] = base;
        co.s2[cls] = base + n;
        co.t1[cls] = base + 2 * n;
        co.t2[cls] = base + 3 * n;
        base += 4 * n;
    }
    count_launch(s);
    k_singular_k1_mixed<<<(unsigned)m.n_touch, MSS_THREADS, 0, s>>>(
        L.geo, m.d_tris, L.pairs, E, N, tab, co, L.mnodes, p.n_steps, g, K1);
    return check_launch("k_singular_k1_mixed");
}

// ---------------------------------- hypersingular operator D^2, mixed ---
// D^{2,d} (eq. D2d) without differencing antiderivatives: blocks 0 and 1 from
// the closed forms alpha F(h) and alpha (F(2h) - 2 F(h)), F(delta) =
// int_0^delta G = erfc(rho / (2 sqrt(alpha delta))) / (4 pi alpha rho); block
// d >= 2 as the hat-weighted time integral of dG/ds (the second difference
// of F is the hat convolution of F'' = dG/ds), by the Gauss nodes of the
// mixed tables: per node the factor of the K tables, with
//   alpha dG/ds = -alpha G / (2 delta) (3 - rho^2 / (2 alpha delta))
//             = -alpha cK (3 + 2 ln2 t) e / w,  t = rho^2 b,  e = exp2(t).
// p1 x p1 weights: the test points' barycentric weights are summed first
// per trial point, the node weights applied per trial point, and the nine
// vertex-pair values of a completed block go out with atomics into D
// (which holds D^1).
constexpr int D2_G = 2;         // intervals per pass over the points
constexpr float TWO_LN2 = 1.3862943611198906f;

// Separated pair (l, j): all blocks of D^2.
__device__ __forceinline__ void regular_pair_d2_mixed(const double *__restrict__ geo,
                                                      const int32_t *__restrict__ tris, int E,
                                                      int N, const float *__restrict__ rule,
                                                      int nq, const float4 *xa,
                                                      const float4 *xl, const float *nd,
                                                      int n_steps, const MixConsts &g,
                                                      float alpha, float *__restrict__ D,
                                                      int l, int j) {
    const int tl[3] = {tris[3 * l], tris[3 * l + 1], tris[3 * l + 2]};
    const int tj[3] = {tris[3 * j], tris[3 * j + 1], tris[3 * j + 2]};
    {
        bool t = false;
        for (int i = 0; i < 3; ++i) t |= (tl[i] == tj[0]) | (tl[i] == tj[1]) | (tl[i] == tj[2]);
        if (t) return;
    }
    const double *gl = geo + (size_t)l * GEO_STRIDE, *gj = geo + (size_t)j * GEO_STRIDE;
    float Dv[3], B1[3], B2[3];
    for (int c = 0; c < 3; ++c) {
        Dv[c] = (float)(gl[GEO_V0 + c] - gj[GEO_V0 + c]);
        B1[c] = (float)(gj[GEO_V1 + c] - gj[GEO_V0 + c]);
        B2[c] = (float)(gj[GEO_V2 + c] - gj[GEO_V1 + c]);
    }
    const double nn = gl[GEO_N] * gj[GEO_N] + gl[GEO_N + 1] * gj[GEO_N + 1] + gl[GEO_N + 2] * gj[GEO_N + 2];
    const float scale = (float)(4.0 * gl[GEO_AREA] * gj[GEO_AREA] * nn);
    const size_t NN = (size_t)N * N;
    auto emit = [&](int d, const float (&v)[9]) {
        float *blk = D + (size_t)d * NN;
#pragma unroll
        for (int va = 0; va < 3; ++va)
#pragma unroll
            for (int vb = 0; vb < 3; ++vb) atomicAdd(blk + (size_t)tl[va] * N + tj[vb], v[3 * va + vb]);
    };
    const float pG = 0.25f / 3.14159265f;  // alpha F = erfc / (4 pi rho)

    // pass 1: blocks 0 and 1 (closed forms) and the k = 1 interval of block 2
    float b0[9], b1[9], b2[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) b0[k] = b1[k] = b2[k] = 0.f;
    for (int b = 0; b < nq; ++b) {
        const float t1 = rule[4 * b], t2 = rule[4 * b + 1], wb = rule[4 * b + 2];
        const float r0b = Dv[0] - (t1 * B1[0] + t2 * B2[0]);
        const float r1b = Dv[1] - (t1 * B1[1] + t2 * B2[1]);
        const float r2b = Dv[2] - (t1 * B1[2] + t2 * B2[2]);
        float s0[3] = {0.f, 0.f, 0.f}, s1[3] = {0.f, 0.f, 0.f}, s2[3] = {0.f, 0.f, 0.f};
        for (int a = 0; a < nq; ++a) {
            const float4 xq = xa[a], lq = xl[a];  // lq: w_a lambda_v(a), v = 0..2
            const float r0 = r0b + xq.x, r1 = r1b + xq.y, r2 = r2b + xq.z;
            const float rr = r0 * r0 + r1 * r1 + r2 * r2;
            const float irho = rsqrtf(rr), rho = rr * irho;
            const float e1 = erfcf(rho * g.c1), e2 = erfcf(rho * g.c2);
            const float f0 = pG * irho * e1, f1 = pG * irho * (e2 - 2.f * e1);
            float f2 = 0.f;
            if (n_steps > 2) {
#pragma unroll
                for (int q = 0; q < MIX_NG1; ++q) {
                    const float4 c = reinterpret_cast<const float4 *>(nd)[q];
                    const float t = rr * c.x;
                    f2 = fmaf(-alpha * c.z * fmaf(TWO_LN2, t, 3.f), ex2(t), f2);
                }
            }
            const float lw[3] = {lq.x, lq.y, lq.z};
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                s0[v] = fmaf(lw[v], f0, s0[v]);
                s1[v] = fmaf(lw[v], f1, s1[v]);
                s2[v] = fmaf(lw[v], f2, s2[v]);
            }
        }
        const float lb[3] = {(1.f - t1) * wb, (t1 - t2) * wb, t2 * wb};
#pragma unroll
        for (int va = 0; va < 3; ++va)
#pragma unroll
            for (int vb = 0; vb < 3; ++vb) {
                b0[3 * va + vb] = fmaf(s0[va], lb[vb], b0[3 * va + vb]);
                b1[3 * va + vb] = fmaf(s1[va], lb[vb], b1[3 * va + vb]);
                b2[3 * va + vb] = fmaf(s2[va], lb[vb], b2[3 * va + vb]);
            }
    }
    float carry[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        b0[k] *= scale;
        b1[k] *= scale;
        carry[k] = scale * b2[k];
    }
    emit(0, b0);
    if (n_steps > 1) emit(1, b1);

    // blocks d >= 2: table chunks of MIX_CH intervals, passes of D2_G
    const float *tab = nd + MIX_K1;
    for (int d0 = 2; d0 < n_steps; d0 += MIX_CH) {
        const int ng = mixed_chunk_ng(d0), ivf = mixed_iv_floats(ng);
        const int n_int = min(MIX_CH, n_steps - d0);
        for (int u0 = 0; u0 < n_int; u0 += D2_G) {
            const float *tg = tab + u0 * ivf;
            float fall[D2_G][9], rise[D2_G][9];
#pragma unroll
            for (int gg = 0; gg < D2_G; ++gg)
#pragma unroll
                for (int k = 0; k < 9; ++k) fall[gg][k] = rise[gg][k] = 0.f;
            for (int b = 0; b < nq; ++b) {
                const float t1 = rule[4 * b], t2 = rule[4 * b + 1], wb = rule[4 * b + 2];
                const float r0b = Dv[0] - (t1 * B1[0] + t2 * B2[0]);
                const float r1b = Dv[1] - (t1 * B1[1] + t2 * B2[1]);
                const float r2b = Dv[2] - (t1 * B1[2] + t2 * B2[2]);
                float C[D2_G][4][3];  // per interval, node, test vertex
#pragma unroll
                for (int gg = 0; gg < D2_G; ++gg)
#pragma unroll
                    for (int q = 0; q < 4; ++q) C[gg][q][0] = C[gg][q][1] = C[gg][q][2] = 0.f;
                for (int a = 0; a < nq; ++a) {
                    const float4 xq = xa[a], lq = xl[a];
                    const float r0 = r0b + xq.x, r1 = r1b + xq.y, r2 = r2b + xq.z;
                    const float rr = r0 * r0 + r1 * r1 + r2 * r2;
#pragma unroll
                    for (int gg = 0; gg < D2_G; ++gg) {
                        const float4 bb = ld_tab<true>(tg + gg * ivf);
                        const float bq[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (q >= ng) break;
                            const float t = rr * bq[q];
                            const float f = fmaf(TWO_LN2, t, 3.f) * ex2(t);
                            C[gg][q][0] = fmaf(lq.x, f, C[gg][q][0]);
                            C[gg][q][1] = fmaf(lq.y, f, C[gg][q][1]);
                            C[gg][q][2] = fmaf(lq.z, f, C[gg][q][2]);
                        }
                    }
                }
                const float lb[3] = {(1.f - t1) * wb, (t1 - t2) * wb, t2 * wb};
#pragma unroll
                for (int gg = 0; gg < D2_G; ++gg) {
                    if (u0 + gg >= n_int) break;
                    float Fa[3] = {0.f, 0.f, 0.f}, Ra[3] = {0.f, 0.f, 0.f};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (q >= ng) break;
                        const float4 c = ld_tab<true>(tg + gg * ivf + 4 + 4 * q);  // (cVf, cKf, cVr, cKr)
#pragma unroll
                        for (int va = 0; va < 3; ++va) {
                            Fa[va] = fmaf(c.y, C[gg][q][va], Fa[va]);
                            Ra[va] = fmaf(c.w, C[gg][q][va], Ra[va]);
                        }
                    }
#pragma unroll
                    for (int va = 0; va < 3; ++va)
#pragma unroll
                        for (int vb = 0; vb < 3; ++vb) {
                            fall[gg][3 * va + vb] = fmaf(Fa[va], lb[vb], fall[gg][3 * va + vb]);
                            rise[gg][3 * va + vb] = fmaf(Ra[va], lb[vb], rise[gg][3 * va + vb]);
                        }
                }
            }
            const float sa = -alpha * scale;
#pragma unroll
            for (int gg = 0; gg < D2_G; ++gg) {
                if (u0 + gg >= n_int) break;
                float v[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    v[k] = fmaf(sa, fall[gg][k], carry[k]);
                    carry[k] = sa * rise[gg][k];
                }
                emit(d0 + u0 + gg, v);
            }
        }
        tab += MIX_CH * ivf;
    }
}

__global__ void __launch_bounds__(MREG_THREADS)
k_regular_d2_mixed(const double *__restrict__ geo, const int32_t *__restrict__ tris, int E, int N,
                   const float *__restrict__ rule, int nq, const float *__restrict__ nodes,
                   int n_nodes_f, int n_steps, MixConsts g, float alpha, float *__restrict__ D) {
    extern __shared__ float smf[];
    float4 *xa = reinterpret_cast<float4 *>(smf);       // x_a - P0_l and w_a
    float4 *xl = xa + MAX_RULE_M;                       // w_a lambda_v(a)
    float *nd = smf + 8 * MAX_RULE_M;                   // time nodes
    const int l = blockIdx.y;
    const int j = blockIdx.x * MREG_THREADS + threadIdx.x;
    load_test_points(geo + (size_t)l * GEO_STRIDE, rule, nq, xa);
    for (int a = threadIdx.x; a < nq; a += MREG_THREADS) {
        const float s1 = rule[4 * a], s2 = rule[4 * a + 1], w = rule[4 * a + 2];
        xl[a] = make_float4((1.f - s1) * w, (s1 - s2) * w, s2 * w, 0.f);
    }
    for (int i = threadIdx.x; i < n_nodes_f; i += MREG_THREADS) nd[i] = nodes[i];
    __syncthreads();
    if (j < E) regular_pair_d2_mixed(geo, tris, E, N, rule, nq, xa, xl, nd, n_steps, g, alpha, D, l, j);
}

// Touching pairs of D^2 in mixed precision: one CTA per unordered pair, the
// difference-form rule for r and the rules' coordinates for the barycentric
// weights; entry (a, b) and, for a != b, the mirrored (b, a) receive the
// same nine values.  Sub-chunks of D2_SCH intervals.
constexpr int D2_SCH = 4;

__global__ void __launch_bounds__(MSS_THREADS)
k_singular_d2_mixed(const double *__restrict__ geo, const int32_t *__restrict__ tris,
                    const TouchPair *__restrict__ pairs, int E, int N, MixSS tab, MixK1Coords co,
                    const float *__restrict__ nodes, int n_steps, MixConsts g, float alpha,
                    float *__restrict__ D) {
    constexpr int S = D2_SCH + 1;
    __shared__ float red[MSS_THREADS / 32][9 * S];
    __shared__ float fin[9 * S];
    const TouchPair P = pairs[blockIdx.x];
    const int a = P.a, b = P.b, cls = P.cls;
    if (a < 0 || b < a || b >= E || cls < PAIR_VERTEX || cls > PAIR_IDENTICAL) return;
    const double *ga = geo + (size_t)a * GEO_STRIDE, *gb = geo + (size_t)b * GEO_STRIDE;
    const int oa[3] = {P.perm & 3, (P.perm >> 2) & 3, (P.perm >> 4) & 3};
    const int ob[3] = {(P.perm >> 6) & 3, (P.perm >> 8) & 3, (P.perm >> 10) & 3};
    float X[4][3];
    for (int c = 0; c < 3; ++c) {
        const double A1 = ga[3 * oa[1] + c] - ga[3 * oa[0] + c], A2 = ga[3 * oa[2] + c] - ga[3 * oa[1] + c];
        const double Bv1 = gb[3 * ob[1] + c] - gb[3 * ob[0] + c], Bv2 = gb[3 * ob[2] + c] - gb[3 * ob[1] + c];
        if (cls == PAIR_IDENTICAL) {
            X[0][c] = (float)-A1; X[1][c] = (float)-A2; X[2][c] = 0.f; X[3][c] = 0.f;
        } else if (cls == PAIR_EDGE) {
            X[0][c] = (float)-A1; X[1][c] = (float)A2; X[2][c] = (float)-Bv2; X[3][c] = 0.f;
        } else {
            X[0][c] = (float)A1; X[1][c] = (float)A2; X[2][c] = (float)-Bv1; X[3][c] = (float)-Bv2;
        }
    }
    int na_node[3], nb_node[3];
    for (int c = 0; c < 3; ++c) {
        na_node[c] = tris[3 * a + oa[c]];
        nb_node[c] = tris[3 * b + ob[c]];
    }
    const double nn = ga[GEO_N] * gb[GEO_N] + ga[GEO_N + 1] * gb[GEO_N + 1] + ga[GEO_N + 2] * gb[GEO_N + 2];
    const float scale = (float)(4.0 * ga[GEO_AREA] * gb[GEO_AREA] * nn);
    const bool ident = cls == PAIR_IDENTICAL;
    const int npt = tab.n[cls];
    const float *R0 = tab.p0[cls], *R1 = tab.p1[cls], *R2 = tab.p2[cls], *R3 = tab.p3[cls],
                *W = tab.w[cls];
    const float *S1 = co.s1[cls], *S2 = co.s2[cls], *T1 = co.t1[cls], *T2 = co.t2[cls];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t NN = (size_t)N * N;
    const float pG = 0.25f / 3.14159265f;

    // point p: r^2 and the nine weights w lambda_va(s) lambda_vb(t)
    auto point = [&](int p, float &rr, float (&wl)[9]) {
        const float q0 = R0[p], q1 = R1[p], q2 = R2[p], q3 = R3[p];
        float r[3];
        for (int c = 0; c < 3; ++c) r[c] = q0 * X[0][c] + q1 * X[1][c] + q2 * X[2][c] + q3 * X[3][c];
        rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        const float w = W[p], s1 = S1[p], s2 = S2[p], t1 = T1[p], t2 = T2[p];
        const float la[3] = {w * (1.f - s1), w * (s1 - s2), w * s2}, lb[3] = {1.f - t1, t1 - t2, t2};
#pragma unroll
        for (int va = 0; va < 3; ++va)
#pragma unroll
            for (int vb = 0; vb < 3; ++vb) wl[3 * va + vb] = la[va] * lb[vb];
    };
    auto reduce = [&](float *vals, int nv) {
        for (int k = 0; k < nv; ++k) {
            float v = vals[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < nv) {
            float sum = 0.f;
            for (int wi = 0; wi < MSS_THREADS / 32; ++wi) sum += red[wi][threadIdx.x];
            fin[threadIdx.x] = scale * sum;
        }
        __syncthreads();
    };
    auto emit = [&](int d, int k, float val) {
        const int va = k / 3, vb = k % 3;
        float *blk = D + (size_t)d * NN;
        atomicAdd(blk + (size_t)na_node[va] * N + nb_node[vb], val);
        if (!ident) atomicAdd(blk + (size_t)nb_node[vb] * N + na_node[va], val);
    };

    // pass 1: blocks 0, 1 and the k = 1 interval of block 2 (27 sums)
    {
        float z[27];
#pragma unroll
        for (int i = 0; i < 27; ++i) z[i] = 0.f;
        for (int p = threadIdx.x; p < npt; p += MSS_THREADS) {
            float rr, wl[9];
            point(p, rr, wl);
            const float irho = rsqrtf(rr), rho = rr * irho;
            const float e1 = erfcf(rho * g.c1), e2 = erfcf(rho * g.c2);
            const float f0 = pG * irho * e1, f1 = pG * irho * (e2 - 2.f * e1);
            float f2 = 0.f;
            if (n_steps > 2) {
#pragma unroll
                for (int q = 0; q < MIX_NG1; ++q) {
                    const float4 c = reinterpret_cast<const float4 *>(nodes)[q];
                    const float t = rr * c.x;
                    f2 = fmaf(-alpha * c.z * fmaf(TWO_LN2, t, 3.f), ex2(t), f2);
                }
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                z[k] = fmaf(wl[k], f0, z[k]);
                z[9 + k] = fmaf(wl[k], f1, z[9 + k]);
                z[18 + k] = fmaf(wl[k], f2, z[18 + k]);
            }
        }
        // reduce in three rounds of nine (fin holds 9 S >= 27 entries)
        reduce(z, 27);
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < 9; ++k) {
            emit(0, k, fin[k]);
            if (n_steps > 1) emit(1, k, fin[9 + k]);
        }
    }
    float carry[9];
    for (int k = 0; k < 9; ++k) carry[k] = fin[18 + k];
    __syncthreads();

    const float *ntab = nodes + MIX_K1;
    for (int d0 = 2; d0 < n_steps; d0 += MIX_CH) {
        const int ng = mixed_chunk_ng(d0), ivf = mixed_iv_floats(ng);
        for (int h0 = 0; h0 < MIX_CH && d0 + h0 < n_steps; h0 += D2_SCH) {
            const int n_int = min(D2_SCH, n_steps - d0 - h0);
            float acc[9 * S];
#pragma unroll
            for (int i = 0; i < 9 * S; ++i) acc[i] = 0.f;
            const float *tb = ntab + h0 * ivf;
            for (int p = threadIdx.x; p < npt; p += MSS_THREADS) {
                float rr, wl[9];
                point(p, rr, wl);
#pragma unroll
                for (int u = 0; u < D2_SCH; ++u) {
                    if (u >= n_int) break;
                    const float4 bb = ld_tab<false>(tb + u * ivf);
                    const float bq[4] = {bb.x, bb.y, bb.z, bb.w};
                    float fall = 0.f, rise = 0.f;
                    for (int q = 0; q < ng; ++q) {
                        const float t = rr * bq[q];
                        const float f = fmaf(TWO_LN2, t, 3.f) * ex2(t);
                        const float4 c = ld_tab<false>(tb + u * ivf + 4 + 4 * q);
                        fall = fmaf(c.y, f, fall);
                        rise = fmaf(c.w, f, rise);
                    }
                    fall *= -alpha;
                    rise *= -alpha;
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        acc[k * S + u] = fmaf(wl[k], fall, acc[k * S + u]);
                        acc[k * S + u + 1] = fmaf(wl[k], rise, acc[k * S + u + 1]);
                    }
                }
            }
            reduce(acc, 9 * S);
            if (threadIdx.x == 0) {
                for (int u = 0; u < n_int; ++u)
                    for (int k = 0; k < 9; ++k)
                        emit(d0 + h0 + u, k, fin[k * S + u] + (u == 0 ? carry[k] : 0.f));
            }
            for (int k = 0; k < 9; ++k) carry[k] = fin[k * S + n_int];
            __syncthreads();
        }
        ntab += MIX_CH * ivf;
    }
}

stb_status run_d2_singular_mixed(const Mesh &m, const stb_params &p, float *D,
                                 const AssemblyLayout &L, const float *coords, cudaStream_t s) {
    if (m.n_touch == 0) return STB_OK;
    const MixConsts g = mix_consts(p);
    const MixSS tab = mix_ss(L);
    MixK1Coords co{};
    const float *base = coords;
    for (int cls = 1; cls <= 3; ++cls) {
        const size_t n = L.ss_n[cls];
        co.s1[cls] = base;
        co.s2[cls] = base + n;
        co.t1[cls] = base + 2 * n;
        co.t2[cls] = base + 3 * n;
        base += 4 * n;
    }
    count_launch(s);
    k_singular_d2_mixed<<<(unsigned)m.n_touch, MSS_THREADS, 0, s>>>(
        L.geo, m.d_tris, L.pairs, (int)m.n_tris, (int)m.n_nodes, tab, co, L.mnodes, p.n_steps, g,
        (float)p.alpha, D);
    return check_launch("k_singular_d2_mixed");
}

stb_status run_d2_regular_mixed(const Mesh &m, const stb_params &p, float *D,
                                const AssemblyLayout &L, cudaStream_t s) {
    const int E = (int)m.n_tris, N = (int)m.n_nodes;
    const int nq = p.quad_regular * p.quad_regular;
    const MixConsts g = mix_consts(p);
    const int nf = (int)mixed_node_floats(p.n_steps);
    const size_t smem = sizeof(float) * (8 * MAX_RULE_M + (size_t)nf);
    STB_CUDA(cudaFuncSetAttribute(k_regular_d2_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    dim3 grid((E + MREG_THREADS - 1) / MREG_THREADS, E);
    count_launch(s);
    k_regular_d2_mixed<<<grid, MREG_THREADS, smem, s>>>(L.geo, m.d_tris, E, N, L.mrule, nq,
                                                         L.mnodes, nf, p.n_steps, g,
                                                         (float)p.alpha, D);
    return check_launch("k_regular_d2_mixed");
}

// ------------------------------------ matrix-free K g (no K storage) ---
// V is stored as by k_regular_mixed; the blocks of K are contracted with the
// Dirichlet data as they are formed, f^k[l] += sum_{d <= k} K^d[l][j]
// g^{k-d}[j], so K is never written (half the memory of the assembly).
// The CTA's row l and 128 columns j: g of those columns sits in shared
// memory (n_steps x nrhs <= VRHS_MAX columns of 128 floats); per completed
// block range and tile of VRHS_KT steps k every thread forms its partial
// products, a warp sums them with shuffles and lane 0 adds them to the row's
// shared sums, which go to f (FP64 atomics) at the end.  Every thread of a
// CTA runs the same loop (touching pairs and the ragged tail contribute
// zero), so the shuffles see full warps.
constexpr int VRHS_MAX = 128;  // n_steps * nrhs
constexpr int VRHS_KT = 8;

// f partial: for the blocks dlo..dlo+cnt-1 (values Kv[u], scaled), all k.
template <int CNT>
__device__ __forceinline__ void vrhs_contract(const float (&Kv)[CNT], int dlo, int cnt,
                                              int n_steps, int nrhs, const float *gs,
                                              float *sf, bool active) {
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < nrhs; ++r) {
        const float *g = gs + (size_t)r * n_steps * MREG_THREADS;  // [i][tid]
        for (int k0 = dlo; k0 < n_steps; k0 += VRHS_KT) {
            float v[VRHS_KT];
#pragma unroll
            for (int t = 0; t < VRHS_KT; ++t) v[t] = 0.f;
            if (active) {
#pragma unroll
                for (int u = 0; u < CNT; ++u) {
                    if (u >= cnt) break;
                    const int d = dlo + u;
#pragma unroll
                    for (int t = 0; t < VRHS_KT; ++t) {
                        const int k = k0 + t;
                        if (k >= d && k < n_steps)
                            v[t] = fmaf(Kv[u], g[(size_t)(k - d) * MREG_THREADS + threadIdx.x], v[t]);
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < VRHS_KT; ++t) {
                float x = v[t];
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == 0 && k0 + t < n_steps) atomicAdd(sf + r * n_steps + k0 + t, x);
            }
        }
    }
}

__global__ void __launch_bounds__(MREG_THREADS)
k_regular_vrhs_mixed(const double *__restrict__ geo, const int32_t *__restrict__ tris, int E,
                     const float *__restrict__ rule, int nq, const float *__restrict__ nodes,
                     int n_nodes_f, int n_steps, MixConsts g, float *__restrict__ V,
                     const double *__restrict__ gd, int nrhs, double *__restrict__ f) {
    extern __shared__ float smf[];
    float4 *xa = reinterpret_cast<float4 *>(smf);
    float *nd = smf + 4 * MAX_RULE_M;
    float *gs = nd + n_nodes_f;                           // [nrhs][n_steps][128]
    float *sf = gs + (size_t)nrhs * n_steps * MREG_THREADS; // [nrhs][n_steps]
    const int l = blockIdx.y;
    const int j = blockIdx.x * MREG_THREADS + threadIdx.x;
    load_test_points(geo + (size_t)l * GEO_STRIDE, rule, nq, xa);
    for (int i = threadIdx.x; i < n_nodes_f; i += MREG_THREADS) nd[i] = nodes[i];
    for (int i = threadIdx.x; i < nrhs * n_steps; i += MREG_THREADS) sf[i] = 0.f;
    for (int ri = 0; ri < nrhs * n_steps; ++ri)  // row (r, i) of g for the CTA's columns
        gs[(size_t)ri * MREG_THREADS + threadIdx.x] =
            j < E ? (float)gd[(size_t)ri * E + j] : 0.f;
    __syncthreads();

    const int jj = j < E ? j : E - 1;
    const int32_t tl[3] = {tris[3 * l], tris[3 * l + 1], tris[3 * l + 2]};
    const int32_t tj[3] = {tris[3 * jj], tris[3 * jj + 1], tris[3 * jj + 2]};
    bool touch = false;
    for (int i = 0; i < 3; ++i) touch |= (tl[i] == tj[0]) | (tl[i] == tj[1]) | (tl[i] == tj[2]);
    const bool active = j < E && !touch;
    // a touching or ragged thread evaluates a separated stand-in pair (its
    // values are discarded) so that every thread runs the same loop
    const int jc = active ? jj : (l + E / 2) % E;
    const double *gl = geo + (size_t)l * GEO_STRIDE, *gj = geo + (size_t)jc * GEO_STRIDE;
    float D[3], B1[3], B2[3], n[3];
    for (int c = 0; c < 3; ++c) {
        D[c] = (float)(gl[GEO_V0 + c] - gj[GEO_V0 + c]);
        B1[c] = (float)(gj[GEO_V1 + c] - gj[GEO_V0 + c]);
        B2[c] = (float)(gj[GEO_V2 + c] - gj[GEO_V1 + c]);
        n[c] = (float)gj[GEO_N + c];
    }
    const float scale = (float)(4.0 * gl[GEO_AREA] * gj[GEO_AREA]);
    const size_t EE = (size_t)E * E, ij = (size_t)l * E + jj;

    float v0 = 0.f, v1 = 0.f, k0 = 0.f, k1 = 0.f, v2 = 0.f, k2 = 0.f;
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
            const float rn = r0 * n[0] + r1 * n[1] + r2 * n[2];
            const float w = xq.w * wb, wrn = w * rn;
            float a0, a1, c0, c1;
            k_d01(rho, irho, g, a0, a1, c0, c1);
            v0 = fmaf(w, a0, v0);
            v1 = fmaf(w, a1, v1);
            k0 = fmaf(wrn, c0, k0);
            k1 = fmaf(wrn, c1, k1);
            if (n_steps > 2) {
#pragma unroll
                for (int q = 0; q < MIX_NG1; ++q) {
                    const float4 c = reinterpret_cast<const float4 *>(nd)[q];
                    const float e = ex2(rr * c.x);
                    v2 = fmaf(w * c.y, e, v2);
                    k2 = fmaf(wrn * c.z, e, k2);
                }
            }
        }
    }
    if (active) {
        V[ij] = scale * v0;
        if (n_steps > 1) V[EE + ij] = scale * v1;
    }
    {
        const float Kv[2] = {scale * k0, scale * k1};
        vrhs_contract<2>(Kv, 0, min(2, n_steps), n_steps, nrhs, gs, sf, active);
    }
    const float *tab = nd + MIX_K1;
    float2 carry = make_float2(v2, k2);
    for (int d0 = 2; d0 < n_steps; d0 += MIX_CH) {
        float2 acc[MIX_CH + 1];
        acc[0] = carry;
#pragma unroll
        for (int u = 1; u <= MIX_CH; ++u) acc[u] = make_float2(0.f, 0.f);
        const int ng = mixed_chunk_ng(d0);
        const int n_pass = (min(MIX_CH, n_steps - d0) + MIX_G - 1) / MIX_G;
        if (ng == 4)
            chunk_sum<4>(tab, n_pass, rule, nq, xa, D, B1, B2, n, acc);
        else if (ng == 3)
            chunk_sum<3>(tab, n_pass, rule, nq, xa, D, B1, B2, n, acc);
        else
            chunk_sum<2>(tab, n_pass, rule, nq, xa, D, B1, B2, n, acc);
        const int cnt = min(MIX_CH, n_steps - d0);
        float Kv[MIX_CH];
#pragma unroll
        for (int u = 0; u < MIX_CH; ++u) {
            Kv[u] = scale * acc[u].y;
            if (active && u < cnt) V[(size_t)(d0 + u) * EE + ij] = scale * acc[u].x;
        }
        vrhs_contract<MIX_CH>(Kv, d0, cnt, n_steps, nrhs, gs, sf, active);
        carry = acc[MIX_CH];
        tab += MIX_CH * mixed_iv_floats(ng);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nrhs * n_steps; i += MREG_THREADS)
        atomicAdd(f + (size_t)i * E + l, (double)sf[i]);
}

// Touching pairs: V of both orders stored, the K blocks of both orders kept
// in shared memory (written by thread 0 of the p0 pair routine) and
// contracted with g by all threads at the end.
template <int CH>
__global__ void __launch_bounds__(MSS_THREADS)
k_singular_vrhs_mixed(const double *__restrict__ geo, const TouchPair *__restrict__ pairs, int E,
                      MixSS tab, const float *__restrict__ nodes, int n_steps, MixConsts g,
                      float *__restrict__ V, const double *__restrict__ gd, int nrhs,
                      double *__restrict__ f) {
    const TouchPair P = pairs[blockIdx.x];
    const int a = P.a, b = P.b;
    if (a < 0 || b < a || b >= E) return;
    __shared__ float kp[2 * VRHS_MAX];
    singular_pair_mixed<CH, float>(geo, P, E, tab, nodes, n_steps, g, V, nullptr, kp);
    __syncthreads();
    if (P.cls == PAIR_IDENTICAL) return;  // K = 0
    const float *kab = kp, *kba = kp + n_steps;
    for (int rk = threadIdx.x; rk < nrhs * n_steps; rk += MSS_THREADS) {
        const int r = rk / n_steps, k = rk % n_steps;
        const double *gr = gd + (size_t)r * n_steps * E;
        double sa = 0.0, sb = 0.0;
        for (int d = 0; d <= k; ++d) {
            sa = fma((double)kab[d], gr[(size_t)(k - d) * E + b], sa);
            sb = fma((double)kba[d], gr[(size_t)(k - d) * E + a], sb);
        }
        atomicAdd(f + ((size_t)r * n_steps + k) * E + a, sa);
        atomicAdd(f + ((size_t)r * n_steps + k) * E + b, sb);
    }
}

// f += (h/2) Delta_l g (the mass part of the right-hand side)
__global__ void k_vrhs_mass(const double *__restrict__ geo, int E, size_t total, double h,
                            const double *__restrict__ gd, double *__restrict__ f) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    f[idx] = fma(0.5 * h * geo[(size_t)(idx % E) * GEO_STRIDE + GEO_AREA], gd[idx], f[idx]);
}

stb_status run_vrhs_mixed(const Mesh &m, const stb_params &p, float *V, const double *gd,
                          int nrhs, double *f, const AssemblyLayout &L, cudaStream_t s) {
    const int E = (int)m.n_tris;
    const int nq = p.quad_regular * p.quad_regular;
    const MixConsts g = mix_consts(p);
    const int nf = (int)mixed_node_floats(p.n_steps);
    const size_t smem = sizeof(float) * (4 * MAX_RULE_M + (size_t)nf +
                                         (size_t)nrhs * p.n_steps * (MREG_THREADS + 1));
    STB_CUDA(cudaFuncSetAttribute(k_regular_vrhs_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    dim3 grid((E + MREG_THREADS - 1) / MREG_THREADS, E);
    count_launch(s);
    k_regular_vrhs_mixed<<<grid, MREG_THREADS, smem, s>>>(L.geo, m.d_tris, E, L.mrule, nq,
                                                           L.mnodes, nf, p.n_steps, g, V, gd, nrhs,
                                                           f);
    stb_status st = check_launch("k_regular_vrhs_mixed");
    if (st) return st;
    if (m.n_touch > 0) {
        const MixSS tab = mix_ss(L);
        count_launch(s);
        k_singular_vrhs_mixed<MIX_CH><<<(unsigned)m.n_touch, MSS_THREADS, 0, s>>>(
            L.geo, L.pairs, E, tab, L.mnodes, p.n_steps, g, V, gd, nrhs, f);
        if ((st = check_launch("k_singular_vrhs_mixed"))) return st;
    }
    const size_t total = (size_t)nrhs * p.n_steps * E;
    count_launch(s);
    k_vrhs_mass<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(L.geo, E, total,
                                                                p.T / p.n_steps, gd, f);
    return check_launch("k_vrhs_mass");
}

// -------------------------------------------------------------- batches ---
// Many independent problems (meshes, alpha, steps) in one persistent launch
// for all their pair classes, mixed precision with FP32 storage.  The work
// items are, first, every touching pair of every problem (the costly items:
// a regularised 4-D rule per pair; put first so that none of them is left
// for the tail), then the separated pairs as (problem, row l, block of NT
// columns), numbered problem by problem.  Every CTA claims items from a
// global counter, so problems of uneven size and step count balance across
// the SMs, and a CTA reloads the time-node table only when its next
// separated-pair item belongs to another problem.
struct BatchDesc {
    const double *geo;
    const int32_t *tris;
    const float *rule, *nodes;
    const TouchPair *pairs;
    float *V, *K;
    MixSS ss;
    MixConsts g;
    long long item0;  // first separated-pair work item of this problem
    int E, nq, n_steps, n_nodes_f, jblocks, touch0, n_touch, pad;
};

// n_touch: touching-pair items (0 to leave them out); n_items: separated-pair
// items; stride > 1 runs every stride-th item only (timing samples).
template <int NT>  // 128 or 256: the touching pairs run on the first 128 threads
__global__ void __launch_bounds__(NT)
k_mixed_batch(const BatchDesc *__restrict__ descs, int n_desc, long long n_touch,
              long long n_items, int stride, unsigned long long *__restrict__ counter) {
    extern __shared__ float smf[];
    float4 *xa = reinterpret_cast<float4 *>(smf);
    float *nd = smf + 4 * MAX_RULE_M;
    __shared__ long long s_item;
    __shared__ int s_prob, s_touch;
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            long long it = (long long)atomicAdd(counter, 1ull) * stride;
            int pr = -1, touch = 0;
            if (it < n_touch) {  // last problem whose first touching pair is <= it
                int lo = 0, hi = n_desc - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (descs[mid].touch0 <= it) lo = mid;
                    else hi = mid - 1;
                }
                pr = lo;
                touch = 1;
            } else if ((it -= n_touch) < n_items) {  // last problem whose first item is <= it
                int lo = 0, hi = n_desc - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (descs[mid].item0 <= it) lo = mid;
                    else hi = mid - 1;
                }
                pr = lo;
            }
            s_item = it;
            s_prob = pr;
            s_touch = touch;
        }
        __syncthreads();
        const long long it = s_item;
        const int pr = s_prob;
        if (pr < 0) break;
        const BatchDesc &D = descs[pr];
        if (s_touch) {
            const int b = (int)(it - D.touch0);
            if (b < D.n_touch) {
                const MixSS ss = D.ss;
                const MixConsts g = D.g;
                singular_pair_mixed<MIX_CH, float, MSS_THREADS>(D.geo, D.pairs[b], D.E, ss, D.nodes,
                                                                D.n_steps, g, D.V, D.K);
            }
            __syncthreads();  // the reduction arrays are reused by the next item
            continue;
        }
        const long long local = it - D.item0;
        const int l = (int)(local / D.jblocks), jb = (int)(local % D.jblocks);
        if (pr != cur) {
            for (int i = threadIdx.x; i < D.n_nodes_f; i += NT) nd[i] = D.nodes[i];
            cur = pr;
        }
        load_test_points(D.geo + (size_t)l * GEO_STRIDE, D.rule, D.nq, xa);
        __syncthreads();
        const int j = jb * NT + threadIdx.x;
        if (j < D.E) {
            const MixConsts g = D.g;
            regular_pair_mixed<float>(D.geo, D.tris, D.E, D.rule, D.nq, xa, nd, D.n_steps, g, D.V,
                                      D.K, l, j);
        }
        __syncthreads();  // shared tables are rewritten by the next item
    }
}

size_t batch_desc_bytes(int n) { return align256((size_t)n * sizeof(BatchDesc)); }

template <int NT>
static stb_status launch_batch_kernel(const BatchDesc *d_descs, int n, long long n_touch,
                                      long long n_items, int stride, unsigned long long *counter,
                                      size_t smem, cudaStream_t s) {
    STB_CUDA(cudaFuncSetAttribute(k_mixed_batch<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    int per_sm = 0, dev = 0, sms = 0;
    STB_CUDA(cudaGetDevice(&dev));
    STB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    STB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mixed_batch<NT>, NT, smem));
    if (per_sm < 1) return fail(STB_ERR_CUDA, "batched kernel does not fit on an SM");
    const long long claims = (n_touch + n_items + stride - 1) / stride;
    const long long grid = std::min<long long>((long long)sms * per_sm, std::max(1LL, claims));
    STB_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
    count_launch(s);
    k_mixed_batch<NT><<<(unsigned)grid, NT, smem, s>>>(d_descs, n, n_touch, n_items, stride, counter);
    return check_launch("k_mixed_batch");
}

// Descriptors of problem i (prepared by prepare_mixed into layouts[i]) for
// work items of `tile` columns; totals for the launch.
static void batch_descs(const Mesh *const *meshes, const stb_params *params,
                        const AssemblyLayout *layouts, float *const *V, float *const *K, int n,
                        int tile, std::vector<BatchDesc> &h, long long &items, int &touch,
                        int &max_nf) {
    h.assign(n, BatchDesc{});
    items = 0;
    touch = 0;
    max_nf = 0;
    for (int i = 0; i < n; ++i) {
        const Mesh &m = *meshes[i];
        const stb_params &p = params[i];
        BatchDesc &D = h[i];
        D.geo = layouts[i].geo;
        D.tris = m.d_tris;
        D.rule = layouts[i].mrule;
        D.nodes = layouts[i].mnodes;
        D.pairs = layouts[i].pairs;
        D.V = V[i];
        D.K = K[i];
        D.ss = mix_ss(layouts[i]);
        D.g = mix_consts(p);
        D.E = (int)m.n_tris;
        D.nq = p.quad_regular * p.quad_regular;
        D.n_steps = p.n_steps;
        D.n_nodes_f = (int)mixed_node_floats(p.n_steps);
        D.jblocks = (D.E + tile - 1) / tile;
        D.item0 = items;
        D.touch0 = touch;
        D.n_touch = (int)m.n_touch;
        items += (long long)D.E * D.jblocks;
        touch += D.n_touch;
        max_nf = std::max(max_nf, D.n_nodes_f);
    }
}

stb_status upload_batch(const Mesh *const *meshes, const stb_params *params,
                        const AssemblyLayout *layouts, float *const *V, float *const *K, int n,
                        BatchDesc *d_descs, int tile, cudaStream_t s) {
    std::vector<BatchDesc> h;
    long long items;
    int touch, max_nf;
    batch_descs(meshes, params, layouts, V, K, n, tile, h, items, touch, max_nf);
    STB_CUDA(cudaMemcpyAsync(d_descs, h.data(), h.size() * sizeof(BatchDesc), cudaMemcpyHostToDevice,
                             s));
    return STB_OK;
}

// One launch (descriptors uploaded by upload_batch with the same tile).
// stride > 1 runs every stride-th work item of the separated pairs and no
// touching pairs (timing samples of the tile tuner).
stb_status launch_batch(const Mesh *const *meshes, const stb_params *params,
                        const AssemblyLayout *layouts, float *const *V, float *const *K, int n,
                        const BatchDesc *d_descs, unsigned long long *counter, int tile, int stride,
                        cudaStream_t s) {
    std::vector<BatchDesc> h;
    long long items;
    int touch, max_nf;
    batch_descs(meshes, params, layouts, V, K, n, tile, h, items, touch, max_nf);
    const size_t smem = sizeof(float) * (4 * MAX_RULE_M + (size_t)max_nf);
    const long long n_touch = stride > 1 ? 0 : touch;
    return tile == 256 ? launch_batch_kernel<256>(d_descs, n, n_touch, items, stride, counter, smem, s)
                       : launch_batch_kernel<128>(d_descs, n, n_touch, items, stride, counter, smem, s);
}

}  // namespace stb
