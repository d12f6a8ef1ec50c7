// stb_potentials.cu -- the discretised representation formula (eq. repr,
// Sec. 3.5): single-layer potential V~ w_h of a piecewise-constant density
// and double-layer potential W u_h of a density piecewise linear in space,
// at points (x, t) off the boundary.
//
// With t = t_k + eps (k = min(floor(t/h), E_t - 1), eps = t - k h in
// [0, h]) the paper writes each potential as a sum over the past steps of
// differences of the temporal antiderivative at d h + eps and (d+1) h + eps,
// plus the current step's difference at 0 and eps.  Summation by parts turns
// this into one antiderivative value per level d = 0..k, weighted by the
// backward differences of the density in time,
//   dw_i = w_i - w_{i-1}  (0-based steps, w_{-1} = 0),
// and the constant 1/(4 pi alpha rho) of G^{dtau}(., 0) drops out of the
// telescoped sum (the weights of a level sum to zero), leaving
//   V~ w_h(x,t) = sum_j int_{gamma_j} 1/(4 pi alpha rho) sum_{d=0}^{k}
//                   dw_{k-d,j} erfc(x_d) ds_y,
//   W u_h(x,t)  = sum_j int_{gamma_j} (r.n_y)/(4 pi rho^3) sum_{d=0}^{k}
//                   du_{k-d}(y) [erfc(x_d) + 2 x_d exp(-x_d^2)/sqrt(pi)] ds_y,
// x_d = rho / (2 sqrt(alpha (d h + eps))) (x_d = infinity, a zero term, at
// delta = 0), du_i(y) the hat-function interpolant of the differences at
// the vertices of gamma_j.  Both forms are free of the cancellation of
// erf(x) near 1 (short times, far pairs) and of the normal-derivative
// bracket near x = 0 (long times).  Every point of a triangle uses the
// q x q conical rule; FP64 throughout.
//
// One thread per (point, trial triangle): the per-point time level k is
// uniform across the CTA, the rule's geometry per thread sits in shared
// memory, the levels run outermost so each density difference is loaded
// once per level, and the CTA's partial sums are added in a fixed order by a
// second kernel (deterministic result).
#include <algorithm>
#include <cmath>
#include <vector>

#include "stb_internal.h"
#include "stb_toeplitz.h"

namespace stb {

constexpr int POT_THREADS = 128;
constexpr int POT_MAX_Q = 5;   // q_space <= 5: at most 25 points per triangle
constexpr int POT_MAXR = 4;    // right-hand sides per pass

// d_i = a_i - a_{i-1} along the steps of [nrhs][n_steps][M] (a_{-1} = 0)
__global__ void k_time_diff(const double *__restrict__ a, int n_steps, int64_t M, size_t total,
                            double *__restrict__ d) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int i = (int)((idx / M) % n_steps);
    d[idx] = i == 0 ? a[idx] : a[idx] - a[idx - M];
}

// erfc(x) and exp(-x^2) for x >= 0 in FP32 for the mixed level values:
// erfc(x) = exp(-x^2) P(t), t = 1 / (1 + 0.7 x), P of degree 11 in t fitted
// to the scaled complementary error function exp(x^2) erfc(x) on [0, 12] in
// relative error (weighted least squares with Lawson's reweighting; the
// table is what fit_erfc.py beside the package prints).  In FP32 Horner form
// P is within 3e-7 of it, and erfc within 4e-7 + 3e-7 x^2 relative (the
// second term the FP32 roundings of -log2(e) x^2 and of the exp2
// approximation, as for exp(-x*x)); the terms where that grows are of order
// exp(-x^2), small in every sum.
__device__ __forceinline__ float erfc_fit(float x, float &ee) {
    constexpr float c[12] = {-2.967891987e-06f, 3.950489759e-01f, 3.929870725e-01f,
                             3.164488971e-01f,  -1.607621554e-03f, 2.811871767e-01f,
                             -1.145935178e+00f, 1.161834598e+00f, -2.941623330e-01f,
                             -2.893261313e-01f, 2.367079258e-01f, -5.318045616e-02f};
    const float t = __frcp_rn(fmaf(0.7f, x, 1.f));
    float P = c[11];
#pragma unroll
    for (int k = 10; k >= 0; --k) P = fmaf(P, t, c[k]);
    float e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-1.4426950408889634f * x * x));
    ee = e;
    return e * P;
}


// Partial sums of one CTA: part[which][r][p][blk] (which 0: single layer,
// 1: double layer).  R: arithmetic of the level values (double, or float
// for the mixed path: x - P0 of the triangle formed in FP64 and rounded
// once, the rule points, erfc and exp in FP32; the products with the
// density differences and all sums over levels stay FP64).
template <class R, bool SLP, bool DLP>
__global__ void __launch_bounds__(POT_THREADS)
k_potentials(const double *__restrict__ geo, const int32_t *__restrict__ tris, int E, int N,
             const double *__restrict__ rule, int nq, const double *__restrict__ pts,
             int64_t n_pts, const double *__restrict__ dw, const double *__restrict__ du,
             int r0, int nr, int nrhs, int n_steps, double h, double T, double alpha,
             double *__restrict__ part, int32_t *__restrict__ status) {
    extern __shared__ __align__(8) unsigned char sm_raw[];
    R *s_rho = reinterpret_cast<R *>(sm_raw);     // [nq][POT_THREADS]
    R *s_cs = s_rho + nq * POT_THREADS;           // 2 Delta w_a / (4 pi alpha rho)
    R *s_cd = s_cs + nq * POT_THREADS;            // 2 Delta w_a (r.n) / (4 pi rho^3)
    __shared__ double s_rule[3 * POT_MAX_Q * POT_MAX_Q];
    __shared__ double red[POT_THREADS / 32][2 * POT_MAXR];
    for (int i = threadIdx.x; i < 3 * nq; i += POT_THREADS) s_rule[i] = rule[i];
    const int nblk = gridDim.x, tid = threadIdx.x;
    const int j = blockIdx.x * POT_THREADS + tid;
    const bool active = j < E;
    const double *gj = geo + (size_t)(active ? j : 0) * GEO_STRIDE;
    const int tv0 = DLP && active ? tris[3 * j] : 0, tv1 = DLP && active ? tris[3 * j + 1] : 0,
              tv2 = DLP && active ? tris[3 * j + 2] : 0;
    const double inv_4pi = 0.25 / 3.14159265358979323846;
    const R two_over_sqrtpi = (R)1.12837916709551257390;
    __syncthreads();

    for (int64_t p = blockIdx.y; p < n_pts; p += gridDim.y) {
        const double x0 = pts[4 * p], x1 = pts[4 * p + 1], x2 = pts[4 * p + 2], t = pts[4 * p + 3];
        const bool valid = t >= 0.0 && t <= T;  // uniform over the CTA; else zero outputs
        if (!valid && tid == 0) atomicCAS(status, 0, STB_ERR_INVALID_ARG);
        int k = valid ? (int)floor(t / h) : 0;
        k = min(max(k, 0), n_steps - 1);
        const double eps = valid ? t - k * h : 0.0;
        // the rule's points on gamma_j, seen from x
        if (active && valid) {
            const double area2 = 2.0 * gj[GEO_AREA];
            if constexpr (sizeof(R) == sizeof(float)) {
                // difference form: x - P0 once in FP64, the rule points in FP32
                float d0[3], e1[3], e2[3], nf[3];
                const double xp[3] = {x0, x1, x2};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    d0[c] = (float)(xp[c] - gj[GEO_V0 + c]);
                    e1[c] = (float)(gj[GEO_V1 + c] - gj[GEO_V0 + c]);
                    e2[c] = (float)(gj[GEO_V2 + c] - gj[GEO_V1 + c]);
                    nf[c] = (float)gj[GEO_N + c];
                }
                const float cwa = (float)(area2 * inv_4pi), cws = (float)(area2 * inv_4pi / alpha);
                for (int a = 0; a < nq; ++a) {
                    const float s1 = (float)s_rule[3 * a], s2 = (float)s_rule[3 * a + 1];
                    const float wa = (float)s_rule[3 * a + 2];
                    float r[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) r[c] = d0[c] - (s1 * e1[c] + s2 * e2[c]);
                    const float rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                    const float irho = rsqrtf(rr);
                    const float rn = r[0] * nf[0] + r[1] * nf[1] + r[2] * nf[2];
                    s_rho[a * POT_THREADS + tid] = rr * irho;
                    s_cs[a * POT_THREADS + tid] = cws * wa * irho;
                    s_cd[a * POT_THREADS + tid] = cwa * wa * rn * irho * irho * irho;
                }
            } else {
                for (int a = 0; a < nq; ++a) {
                    const double s1 = s_rule[3 * a], s2 = s_rule[3 * a + 1], wa = s_rule[3 * a + 2];
                    const double xp[3] = {x0, x1, x2};
                    double r[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        r[c] = xp[c] - (gj[GEO_V0 + c] + s1 * (gj[GEO_V1 + c] - gj[GEO_V0 + c]) +
                                        s2 * (gj[GEO_V2 + c] - gj[GEO_V1 + c]));
                    const double rho = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                    const double rn = r[0] * gj[GEO_N] + r[1] * gj[GEO_N + 1] + r[2] * gj[GEO_N + 2];
                    s_rho[a * POT_THREADS + tid] = (R)rho;
                    s_cs[a * POT_THREADS + tid] = (R)(area2 * wa * inv_4pi / (alpha * rho));
                    s_cd[a * POT_THREADS + tid] = (R)(area2 * wa * inv_4pi * rn / (rho * rho * rho));
                }
            }
        }
        double acc_s[POT_MAXR], acc_d[POT_MAXR];
#pragma unroll
        for (int r = 0; r < POT_MAXR; ++r) acc_s[r] = acc_d[r] = 0.0;
        if (active && valid) {
            for (int d = 0; d <= k; ++d) {
                const double delta = d * h + eps;
                if (delta <= 0.0) continue;  // x_d = infinity: zero terms
                R ix;  // 1 / (2 sqrt(alpha delta)), in the level arithmetic
                if constexpr (sizeof(R) == sizeof(float))
                    ix = 0.5f * rsqrtf((float)(alpha * delta));
                else
                    ix = 0.5 / sqrt(alpha * delta);
                R L = 0, L1[3] = {0, 0, 0};
                for (int a = 0; a < nq; ++a) {
                    const R x = s_rho[a * POT_THREADS + tid] * ix;
                    R e, ee = 0;  // erfc(x), exp(-x^2) (double layer only)
                    if constexpr (sizeof(R) == sizeof(float)) {
                        e = erfc_fit(x, ee);
                    } else {
                        e = erfc(x);
                        if (DLP) ee = exp(-x * x);
                    }
                    if (SLP) L = fma(s_cs[a * POT_THREADS + tid], e, L);
                    if (DLP) {
                        const R g = fma(two_over_sqrtpi * x, ee, e);
                        const R c = s_cd[a * POT_THREADS + tid] * g;
                        const R s1 = (R)s_rule[3 * a], s2 = (R)s_rule[3 * a + 1];
                        L1[0] = fma((R)1 - s1, c, L1[0]);
                        L1[1] = fma(s1 - s2, c, L1[1]);
                        L1[2] = fma(s2, c, L1[2]);
                    }
                }
                const int i = k - d;  // step of the density difference
#pragma unroll
                for (int r = 0; r < POT_MAXR; ++r) {
                    if (r >= nr) break;
                    const size_t row = ((size_t)(r0 + r) * n_steps + i);
                    if (SLP) acc_s[r] = fma(__ldg(dw + row * E + j), (double)L, acc_s[r]);
                    if (DLP) {
                        const double *ur = du + row * N;
                        acc_d[r] = fma(__ldg(ur + tv0), (double)L1[0], acc_d[r]);
                        acc_d[r] = fma(__ldg(ur + tv1), (double)L1[1], acc_d[r]);
                        acc_d[r] = fma(__ldg(ur + tv2), (double)L1[2], acc_d[r]);
                    }
                }
            }
        }
        // CTA reduction, fixed order
        const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
        for (int r = 0; r < POT_MAXR; ++r) {
            double a = acc_s[r], b = acc_d[r];
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_xor_sync(0xffffffffu, a, o);
                b += __shfl_xor_sync(0xffffffffu, b, o);
            }
            if (lane == 0) {
                red[warp][2 * r] = a;
                red[warp][2 * r + 1] = b;
            }
        }
        __syncthreads();
        if (tid < 2 * nr) {
            double s = 0.0;
            for (int w = 0; w < POT_THREADS / 32; ++w) s += red[w][tid];
            const int r = r0 + (tid >> 1), which = tid & 1;
            part[(((size_t)which * nrhs + r) * n_pts + p) * nblk + blockIdx.x] = s;
        }
        __syncthreads();
    }
}

// out[r][p] = sum over the CTA partials (fixed order)
__global__ void k_potentials_reduce(const double *__restrict__ part, int nblk, size_t n,
                                    double *__restrict__ slp, double *__restrict__ dlp) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // (r, p)
    if (idx >= n) return;
    if (slp) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part[idx * nblk + b];
        slp[idx] = s;
    }
    if (dlp) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part[(n + idx) * nblk + b];
        dlp[idx] = s;
    }
}

struct PotLayout {
    double *geo, *rule, *dw, *du, *part;
    size_t bytes;
};

static PotLayout pot_layout(const Mesh &m, int n_steps, int nrhs, int64_t n_pts, int q, bool slp,
                            bool dlp, void *ws, size_t cap) {
    Carve c(ws, cap);
    PotLayout L{};
    const int nblk = (int)((m.n_tris + POT_THREADS - 1) / POT_THREADS);
    L.geo = c.take<double>((size_t)m.n_tris * GEO_STRIDE);
    L.rule = c.take<double>(3 * (size_t)q * q);
    L.dw = slp ? c.take<double>((size_t)nrhs * n_steps * m.n_tris) : nullptr;
    L.du = dlp ? c.take<double>((size_t)nrhs * n_steps * m.n_nodes) : nullptr;
    L.part = c.take<double>(2 * (size_t)nrhs * n_pts * nblk);
    L.bytes = c.off;
    return L;
}

static stb_status pot_check(const stb_mesh *mesh, const stb_params *p, int32_t nrhs, int64_t n_pts,
                            int32_t q) {
    if (!mesh || !p) return fail(STB_ERR_INVALID_ARG, "mesh and params must be given");
    if (!(p->alpha > 0) || !(p->T > 0) || p->n_steps < 1)
        return fail(STB_ERR_INVALID_ARG, "alpha, T and n_steps must be positive");
    if (nrhs < 1 || n_pts < 1 || q < 1 || q > POT_MAX_Q)
        return fail(STB_ERR_INVALID_ARG, "need nrhs >= 1, n_pts >= 1, 1 <= q_space <= %d",
                    POT_MAX_Q);
    return STB_OK;
}

// ------------------------------------------------ points x all steps ---
// For points x_p evaluated at every t_k + eps (k = 0..E_t-1, one eps), the
// level values do not depend on k: the potentials are block-Toeplitz
// products
//   V~ w_h(x_p, t_k + eps) = sum_{d=0}^{k} sum_j Ls^d[p][j] dw_{k-d,j},
//   W u_h(x_p, t_k + eps)  = sum_{d=0}^{k} sum_i Ld^d[p][i] du_{k-d,i},
// with the level blocks (delta_d = d h + eps)
//   Ls^d[p][j] = int_{gamma_j} erfc(x_d) / (4 pi alpha rho) ds_y,
//   Ld^d[p][i] = sum_{j around i} int_{gamma_j} phi_i (r.n_y)/(4 pi rho^3)
//                [erfc(x_d) + 2 x_d exp(-x_d^2)/sqrt(pi)] ds_y,
// so every antiderivative is evaluated once per (point, triangle, rule
// point, level) instead of once per evaluation time.  One thread per
// (point, triangle); Ls is stored directly, Ld is added per node with
// atomics (it starts at zero).
template <bool SLP, bool DLP>
__global__ void __launch_bounds__(POT_THREADS)
k_potential_levels(const double *__restrict__ geo, const int32_t *__restrict__ tris, int E, int N,
                   const double *__restrict__ rule, int nq, const double *__restrict__ pts3,
                   int P, int n_steps, double h, double eps, double alpha,
                   double *__restrict__ Ls, double *__restrict__ Ld) {
    extern __shared__ double sm[];
    double *s_rho = sm, *s_cs = s_rho + nq * POT_THREADS, *s_cd = s_cs + nq * POT_THREADS;
    __shared__ double s_rule[3 * POT_MAX_Q * POT_MAX_Q];
    for (int i = threadIdx.x; i < 3 * nq; i += POT_THREADS) s_rule[i] = rule[i];
    __syncthreads();
    const int tid = threadIdx.x, j = blockIdx.x * POT_THREADS + tid;
    const int p = blockIdx.y;
    if (j >= E) return;
    const double *gj = geo + (size_t)j * GEO_STRIDE;
    const double inv_4pi = 0.25 / 3.14159265358979323846;
    const double two_over_sqrtpi = 1.12837916709551257390;
    const double xp[3] = {pts3[3 * (size_t)p], pts3[3 * (size_t)p + 1], pts3[3 * (size_t)p + 2]};
    const double area2 = 2.0 * gj[GEO_AREA];
    for (int a = 0; a < nq; ++a) {
        const double s1 = s_rule[3 * a], s2 = s_rule[3 * a + 1], wa = s_rule[3 * a + 2];
        double r[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            r[c] = xp[c] - (gj[GEO_V0 + c] + s1 * (gj[GEO_V1 + c] - gj[GEO_V0 + c]) +
                            s2 * (gj[GEO_V2 + c] - gj[GEO_V1 + c]));
        const double rho = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        const double rn = r[0] * gj[GEO_N] + r[1] * gj[GEO_N + 1] + r[2] * gj[GEO_N + 2];
        s_rho[a * POT_THREADS + tid] = rho;
        s_cs[a * POT_THREADS + tid] = area2 * wa * inv_4pi / (alpha * rho);
        s_cd[a * POT_THREADS + tid] = area2 * wa * inv_4pi * rn / (rho * rho * rho);
    }
    const int t0 = DLP ? tris[3 * j] : 0, t1 = DLP ? tris[3 * j + 1] : 0,
              t2 = DLP ? tris[3 * j + 2] : 0;
    for (int d = 0; d < n_steps; ++d) {
        const double delta = d * h + eps;
        double L = 0.0, L1[3] = {0.0, 0.0, 0.0};
        if (delta > 0.0) {
            const double ix = 0.5 / sqrt(alpha * delta);
            for (int a = 0; a < nq; ++a) {
                const double x = s_rho[a * POT_THREADS + tid] * ix;
                const double e = erfc(x);
                if (SLP) L = fma(s_cs[a * POT_THREADS + tid], e, L);
                if (DLP) {
                    const double c = s_cd[a * POT_THREADS + tid] *
                                     fma(two_over_sqrtpi * x, exp(-x * x), e);
                    const double s1 = s_rule[3 * a], s2 = s_rule[3 * a + 1];
                    L1[0] = fma(1.0 - s1, c, L1[0]);
                    L1[1] = fma(s1 - s2, c, L1[1]);
                    L1[2] = fma(s2, c, L1[2]);
                }
            }
        }
        const size_t blk = (size_t)d * P + p;
        if (SLP) Ls[blk * E + j] = L;
        if (DLP) {
            double *row = Ld + blk * N;
            atomicAdd(row + t0, L1[0]);
            atomicAdd(row + t1, L1[1]);
            atomicAdd(row + t2, L1[2]);
        }
    }
}

// The same level blocks from FP32 quadrature points (params->precision =
// STB_PREC_MIXED): x - P0 of the triangle formed in FP64 and rounded once,
// the rule points and the level loop in FP32 (erfc and exp of x_d;
// both terms of the double-layer bracket are positive, so nothing cancels),
// Ls is stored FP32 and Ld accumulated per node with FP32 atomics.
template <bool SLP, bool DLP>
__global__ void __launch_bounds__(POT_THREADS)
k_potential_levels_mixed(const double *__restrict__ geo, const int32_t *__restrict__ tris, int E,
                         int N, const double *__restrict__ rule, int nq,
                         const double *__restrict__ pts3, int P, int n_steps, double h, double eps,
                         double alpha, float *__restrict__ Ls, float *__restrict__ Ld) {
    extern __shared__ float smf[];
    float *s_rho = smf, *s_cs = s_rho + nq * POT_THREADS, *s_cd = s_cs + nq * POT_THREADS;
    __shared__ float s_lam[2 * POT_MAX_Q * POT_MAX_Q];
    for (int i = threadIdx.x; i < nq; i += POT_THREADS) {
        s_lam[2 * i] = (float)rule[3 * i];
        s_lam[2 * i + 1] = (float)rule[3 * i + 1];
    }
    __syncthreads();
    const int tid = threadIdx.x, j = blockIdx.x * POT_THREADS + tid;
    const int p = blockIdx.y;
    if (j >= E) return;
    const double *gj = geo + (size_t)j * GEO_STRIDE;
    const double inv_4pi = 0.25 / 3.14159265358979323846;
    const float two_over_sqrtpi = 1.12837916709551257390f;
    const double xp[3] = {pts3[3 * (size_t)p], pts3[3 * (size_t)p + 1], pts3[3 * (size_t)p + 2]};
    const double area2 = 2.0 * gj[GEO_AREA];
    // difference form: x - P0 once in FP64, the rule points in FP32
    float d0[3], e1[3], e2[3], nf[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        d0[c] = (float)(xp[c] - gj[GEO_V0 + c]);
        e1[c] = (float)(gj[GEO_V1 + c] - gj[GEO_V0 + c]);
        e2[c] = (float)(gj[GEO_V2 + c] - gj[GEO_V1 + c]);
        nf[c] = (float)gj[GEO_N + c];
    }
    const float cwa = (float)(area2 * inv_4pi), cws = (float)(area2 * inv_4pi / alpha);
    for (int a = 0; a < nq; ++a) {
        const float s1 = (float)rule[3 * a], s2 = (float)rule[3 * a + 1], wa = (float)rule[3 * a + 2];
        float r[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) r[c] = d0[c] - (s1 * e1[c] + s2 * e2[c]);
        const float rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        const float irho = rsqrtf(rr);
        const float rn = r[0] * nf[0] + r[1] * nf[1] + r[2] * nf[2];
        s_rho[a * POT_THREADS + tid] = rr * irho;
        s_cs[a * POT_THREADS + tid] = cws * wa * irho;
        s_cd[a * POT_THREADS + tid] = cwa * wa * rn * irho * irho * irho;
    }
    const int t0 = DLP ? tris[3 * j] : 0, t1 = DLP ? tris[3 * j + 1] : 0,
              t2 = DLP ? tris[3 * j + 2] : 0;
    for (int d = 0; d < n_steps; ++d) {
        const double delta = d * h + eps;
        float L = 0.f, L1[3] = {0.f, 0.f, 0.f};
        if (delta > 0.0) {
            const float ix = 0.5f * rsqrtf((float)(alpha * delta));  // FP32, as the levels
            for (int a = 0; a < nq; ++a) {
                const float x = s_rho[a * POT_THREADS + tid] * ix;
                float ee;  // exp(-x^2)
                const float e = erfc_fit(x, ee);
                if (SLP) L = fmaf(s_cs[a * POT_THREADS + tid], e, L);
                if (DLP) {
                    const float c = s_cd[a * POT_THREADS + tid] *
                                    fmaf(two_over_sqrtpi * x, ee, e);
                    const float l1 = s_lam[2 * a], l2 = s_lam[2 * a + 1];
                    L1[0] = fmaf(1.f - l1, c, L1[0]);
                    L1[1] = fmaf(l1 - l2, c, L1[1]);
                    L1[2] = fmaf(l2, c, L1[2]);
                }
            }
        }
        const size_t blk = (size_t)d * P + p;
        if (SLP) Ls[blk * E + j] = L;
        if (DLP) {
            float *row = Ld + blk * N;
            atomicAdd(row + t0, L1[0]);
            atomicAdd(row + t1, L1[1]);
            atomicAdd(row + t2, L1[2]);
        }
    }
}

}  // namespace stb

using namespace stb;

extern "C" stb_status stb_potentials_workspace_size(const stb_mesh *mesh, const stb_params *p,
                                                    int32_t nrhs, int64_t n_pts, int32_t q,
                                                    size_t *bytes) {
    stb_status st = pot_check(mesh, p, nrhs, n_pts, q);
    if (st) return st;
    if (!bytes) return fail(STB_ERR_INVALID_ARG, "bytes must be given");
    *bytes = align256(pot_layout(mesh->m, p->n_steps, nrhs, n_pts, q, true, true, nullptr, 0).bytes);
    return STB_OK;
}

extern "C" stb_status stb_potentials(const stb_mesh *mesh, const stb_params *p, const double *points,
                                     int64_t n_pts, const double *w, const double *u1, int32_t nrhs,
                                     int32_t q, double *slp, double *dlp, void *ws,
                                     size_t ws_bytes, stb_stream stream) {
    stb_status st = pot_check(mesh, p, nrhs, n_pts, q);
    if (st) return st;
    if (!points) return fail(STB_ERR_INVALID_ARG, "points must be given");
    if (!slp && !dlp) return fail(STB_ERR_INVALID_ARG, "need slp or dlp");
    if ((slp && !w) || (dlp && !u1))
        return fail(STB_ERR_INVALID_ARG, "slp needs w, dlp needs u1");
    const Mesh &m = mesh->m;
    const bool do_s = slp != nullptr, do_d = dlp != nullptr;
    PotLayout L = pot_layout(m, p->n_steps, nrhs, n_pts, q, do_s, do_d, ws, ws_bytes);
    size_t need;
    if ((st = stb_potentials_workspace_size(mesh, p, nrhs, n_pts, q, &need))) return st;
    if ((st = check_workspace(ws, ws_bytes, need))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    std::vector<double> s1, s2, wr, host;
    triangle_rule(q, s1, s2, wr);
    for (size_t a = 0; a < wr.size(); ++a) {
        host.push_back(s1[a]);
        host.push_back(s2[a]);
        host.push_back(wr[a]);
    }
    STB_CUDA(cudaMemcpyAsync(L.rule, host.data(), host.size() * sizeof(double),
                             cudaMemcpyHostToDevice, s));
    if ((st = launch_geometry(m, L.geo, s))) return st;
    const int n = p->n_steps;
    if (do_s) {
        const size_t tot = (size_t)nrhs * n * m.n_tris;
        count_launch(s);
        k_time_diff<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(w, n, m.n_tris, tot, L.dw);
        if ((st = check_launch("k_time_diff"))) return st;
    }
    if (do_d) {
        const size_t tot = (size_t)nrhs * n * m.n_nodes;
        count_launch(s);
        k_time_diff<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(u1, n, m.n_nodes, tot, L.du);
        if ((st = check_launch("k_time_diff"))) return st;
    }
    const int nq = q * q, nblk = (int)((m.n_tris + POT_THREADS - 1) / POT_THREADS);
    const bool mixed = p->precision == STB_PREC_MIXED;
    dim3 grid((unsigned)nblk, (unsigned)std::min<int64_t>(n_pts, 65535));
    const double h = p->T / n;
    for (int r0 = 0; r0 < nrhs; r0 += POT_MAXR) {
        const int nr = std::min(POT_MAXR, nrhs - r0);
        count_launch(s);
        auto go = [&](auto kern, size_t rsize) -> stb_status {
            const size_t smem = rsize * 3 * nq * POT_THREADS;
            STB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
            kern<<<grid, POT_THREADS, smem, s>>>(L.geo, m.d_tris, (int)m.n_tris, (int)m.n_nodes,
                                                 L.rule, nq, points, n_pts, L.dw, L.du, r0, nr,
                                                 nrhs, n, h, p->T, p->alpha, L.part,
                                                 status_word(ws));
            return STB_OK;
        };
        if (mixed)
            st = do_s && do_d ? go(k_potentials<float, true, true>, sizeof(float))
                 : do_s       ? go(k_potentials<float, true, false>, sizeof(float))
                              : go(k_potentials<float, false, true>, sizeof(float));
        else
            st = do_s && do_d ? go(k_potentials<double, true, true>, sizeof(double))
                 : do_s       ? go(k_potentials<double, true, false>, sizeof(double))
                              : go(k_potentials<double, false, true>, sizeof(double));
        if (st) return st;
        if ((st = check_launch(mixed ? "k_potentials_mixed" : "k_potentials"))) return st;
    }
    const size_t tot = (size_t)nrhs * n_pts;
    count_launch(s);
    k_potentials_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(L.part, nblk, tot, slp, dlp);
    return check_launch("k_potentials_reduce");
}

// ------------------------------------------------ points x all steps ---
namespace stb {
struct GridLayout {
    double *geo, *rule, *dw, *du, *Ls, *Ld, *part;
    size_t bytes;
};

static GridLayout grid_layout(const Mesh &m, int n_steps, int nrhs, int64_t P, int q, bool slp,
                              bool dlp, void *ws, size_t cap) {
    Carve c(ws, cap);
    GridLayout L{};
    L.geo = c.take<double>((size_t)m.n_tris * GEO_STRIDE);
    L.rule = c.take<double>(3 * (size_t)q * q);
    L.dw = slp ? c.take<double>((size_t)nrhs * n_steps * m.n_tris) : nullptr;
    L.du = dlp ? c.take<double>((size_t)nrhs * n_steps * m.n_nodes) : nullptr;
    L.Ls = slp ? c.take<double>((size_t)n_steps * P * m.n_tris) : nullptr;
    L.Ld = dlp ? c.take<double>((size_t)n_steps * P * m.n_nodes) : nullptr;
    // FP64 products (FP64 level blocks) or double-float products (FP32 ones)
    const size_t prod = std::max(toeplitz_partial_bytes(P, n_steps, nrhs),
                                 toeplitz_df_rect_bytes(P, std::max<int64_t>(m.n_tris, m.n_nodes),
                                                        n_steps, nrhs));
    L.part = reinterpret_cast<double *>(c.take<char>(prod));
    L.bytes = c.off;
    return L;
}

template <bool SLP, bool DLP>
static stb_status launch_levels(const Mesh &m, const GridLayout &L, int nq, const double *pts3,
                                int P, int n, double h, double eps, double alpha, bool mixed,
                                cudaStream_t s) {
    dim3 grid((unsigned)((m.n_tris + POT_THREADS - 1) / POT_THREADS), (unsigned)P);
    if (mixed) {
        const size_t smem = sizeof(float) * 3 * nq * POT_THREADS;
        STB_CUDA(cudaFuncSetAttribute(k_potential_levels_mixed<SLP, DLP>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        count_launch(s);
        k_potential_levels_mixed<SLP, DLP><<<grid, POT_THREADS, smem, s>>>(
            L.geo, m.d_tris, (int)m.n_tris, (int)m.n_nodes, L.rule, nq, pts3, P, n, h, eps, alpha,
            reinterpret_cast<float *>(L.Ls), reinterpret_cast<float *>(L.Ld));
        return check_launch("k_potential_levels_mixed");
    }
    const size_t smem = sizeof(double) * 3 * nq * POT_THREADS;
    STB_CUDA(cudaFuncSetAttribute(k_potential_levels<SLP, DLP>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    count_launch(s);
    k_potential_levels<SLP, DLP><<<grid, POT_THREADS, smem, s>>>(
        L.geo, m.d_tris, (int)m.n_tris, (int)m.n_nodes, L.rule, nq, pts3, P, n, h, eps, alpha,
        L.Ls, L.Ld);
    return check_launch("k_potential_levels");
}
}  // namespace stb

extern "C" stb_status stb_potentials_grid_workspace_size(const stb_mesh *mesh, const stb_params *p,
                                                         int32_t nrhs, int64_t n_pts, int32_t q,
                                                         size_t *bytes) {
    stb_status st = pot_check(mesh, p, nrhs, n_pts, q);
    if (st) return st;
    if (!bytes) return fail(STB_ERR_INVALID_ARG, "bytes must be given");
    if (n_pts > 65535) return fail(STB_ERR_INVALID_ARG, "n_pts must be <= 65535 per call");
    *bytes = align256(grid_layout(mesh->m, p->n_steps, nrhs, n_pts, q, true, true, nullptr, 0).bytes);
    return STB_OK;
}

extern "C" stb_status stb_potentials_grid(const stb_mesh *mesh, const stb_params *p,
                                          const double *points3, int64_t n_pts, double eps,
                                          const double *w, const double *u1, int32_t nrhs,
                                          int32_t q, double *slp, double *dlp, void *ws,
                                          size_t ws_bytes, stb_stream stream) {
    size_t need;
    stb_status st = stb_potentials_grid_workspace_size(mesh, p, nrhs, n_pts, q, &need);
    if (st) return st;
    if (!points3) return fail(STB_ERR_INVALID_ARG, "points must be given");
    if (!slp && !dlp) return fail(STB_ERR_INVALID_ARG, "need slp or dlp");
    if ((slp && !w) || (dlp && !u1))
        return fail(STB_ERR_INVALID_ARG, "slp needs w, dlp needs u1");
    const int n = p->n_steps;
    const double h = p->T / n;
    if (!(eps >= 0.0 && eps <= h)) return fail(STB_ERR_INVALID_ARG, "need 0 <= eps <= T / n_steps");
    if ((st = check_workspace(ws, ws_bytes, need))) return st;
    const Mesh &m = mesh->m;
    const bool do_s = slp != nullptr, do_d = dlp != nullptr;
    GridLayout L = grid_layout(m, n, nrhs, n_pts, q, do_s, do_d, ws, ws_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    std::vector<double> s1, s2, wr, host;
    triangle_rule(q, s1, s2, wr);
    for (size_t a = 0; a < wr.size(); ++a) {
        host.push_back(s1[a]);
        host.push_back(s2[a]);
        host.push_back(wr[a]);
    }
    STB_CUDA(cudaMemcpyAsync(L.rule, host.data(), host.size() * sizeof(double),
                             cudaMemcpyHostToDevice, s));
    if ((st = launch_geometry(m, L.geo, s))) return st;
    const int P = (int)n_pts, nq = q * q;
    const bool mixed = p->precision == STB_PREC_MIXED;
    const int32_t lv_store = mixed ? STB_STORE_F32 : STB_STORE_F64;  // level blocks
    if (do_d)
        STB_CUDA(cudaMemsetAsync(L.Ld, 0, (mixed ? sizeof(float) : sizeof(double)) * (size_t)n * P *
                                              m.n_nodes, s));
    if (do_s && do_d)
        st = launch_levels<true, true>(m, L, nq, points3, P, n, h, eps, p->alpha, mixed, s);
    else if (do_s)
        st = launch_levels<true, false>(m, L, nq, points3, P, n, h, eps, p->alpha, mixed, s);
    else
        st = launch_levels<false, true>(m, L, nq, points3, P, n, h, eps, p->alpha, mixed, s);
    if (st) return st;
    if (do_s) {
        const size_t tot = (size_t)nrhs * n * m.n_tris;
        count_launch(s);
        k_time_diff<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(w, n, m.n_tris, tot, L.dw);
        if ((st = check_launch("k_time_diff"))) return st;
        st = mixed ? toeplitz_df_rect(reinterpret_cast<const float *>(L.Ls), P, m.n_tris, n, nrhs,
                                      L.dw, slp, L.part, s)
                   : toeplitz_fp64_rect(L.Ls, lv_store, P, m.n_tris, n, nrhs, L.dw, 0.0, slp,
                                        L.part, s);
        if (st) return st;
    }
    if (do_d) {
        const size_t tot = (size_t)nrhs * n * m.n_nodes;
        count_launch(s);
        k_time_diff<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(u1, n, m.n_nodes, tot, L.du);
        if ((st = check_launch("k_time_diff"))) return st;
        st = mixed ? toeplitz_df_rect(reinterpret_cast<const float *>(L.Ld), P, m.n_nodes, n, nrhs,
                                      L.du, dlp, L.part, s)
                   : toeplitz_fp64_rect(L.Ld, lv_store, P, m.n_nodes, n, nrhs, L.du, 0.0, dlp,
                                        L.part, s);
        if (st) return st;
    }
    return STB_OK;
}
