// stb_dirichlet.cu -- Dirichlet data of exterior heat sources, its L2
// projection into piecewise constants, the right-hand side
// f = (1/2 M_h + K_h) g and the L2(Sigma_h) error of the Neumann datum
// (Sec. 3.4, Sec. 6.1).  One thread per space-time element (r, k, j); the
// space rule (conical, q x q) and time rule (Gauss, n_time) live in shared
// memory.
#include <cmath>
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "stb_dense.h"
#include "stb_heat.h"
#include "stb_internal.h"
#include "stb_nonuniform.h"
#include "stb_toeplitz.h"

namespace stb {

constexpr int DIR_THREADS = 128;
constexpr int MAX_QS = 32;   // q_space <= 32
constexpr int MAX_NT = 64;   // n_time <= 64
constexpr int MAX_SRC = 64;  // sources per right-hand side


struct DirLayout {
    double *geo, *rule, *src, *part;
    size_t bytes;
};

static DirLayout dir_layout(const Mesh &m, int nrhs, int n_src, int q, int nt, void *ws,
                            size_t cap, size_t n_part) {
    Carve c(ws, cap);
    DirLayout L{};
    L.geo = c.take<double>((size_t)m.n_tris * GEO_STRIDE);
    L.rule = c.take<double>(3 * (size_t)q * q + 2 * (size_t)nt);
    L.src = c.take<double>(5 * (size_t)nrhs * n_src);
    L.part = c.take<double>(n_part);
    L.bytes = c.off;
    return L;
}

static void host_rules(int q, int nt, std::vector<double> &out) {
    std::vector<double> s1, s2, w, tx(nt), tw(nt);
    triangle_rule(q, s1, s2, w);
    gauss_legendre01(nt, tx.data(), tw.data());
    out.clear();
    for (size_t i = 0; i < w.size(); ++i) {
        out.push_back(s1[i]);
        out.push_back(s2[i]);
        out.push_back(w[i]);
    }
    out.insert(out.end(), tx.begin(), tx.end());
    out.insert(out.end(), tw.begin(), tw.end());
}

// g_{r,k,j} = (h Delta_j)^{-1} int_{t_k}^{t_{k+1}} int_{gamma_j} g_r  (element mean);
// NEU: of the Neumann datum w_r = alpha du_r/dn_x = -sum_s weight_s G (x - y_s).n_x
// / (2 (t - t0_s)) instead of the Dirichlet datum
// FP32 fast path for one source per right-hand side (uniform steps): the
// time-node factors of the heat kernel (1/(4 alpha tau), (4 pi alpha tau)^-3/2)
// depend on the time node only, so the sums run time nodes outside and rule
// points inside, x - y* in difference form (P0 - y* in FP64 once, rounded,
// plus the edge vectors in FP32).  Returns, for the triangle's row of nodes,
// sum_b tw_b c_b sum_a w_a f_a(b) with f = exp(-r^2 / (4 alpha tau)) (MODE 0,
// the projection) or the error sums of the Neumann datum (MODE 1).
struct OneSourceGeom {
    float p[3], e1[3], e2[3];
};
__device__ __forceinline__ OneSourceGeom one_source_geom(const double *gj, const float *S) {
    OneSourceGeom G;
    for (int c = 0; c < 3; ++c) {
        G.p[c] = (float)(gj[c] - (double)S[c]);
        G.e1[c] = (float)(gj[3 + c] - gj[c]);
        G.e2[c] = (float)(gj[6 + c] - gj[3 + c]);
    }
    return G;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(x));
    return e;
}

template <class R, bool NEU = false>
__global__ void __launch_bounds__(DIR_THREADS)
k_project(const double *__restrict__ geo, int E, const double *__restrict__ rule, int nq, int nt,
          const double *__restrict__ src, int n_src, int nrhs, int n_steps, double h_, double alpha_,
          double *__restrict__ g, const double *__restrict__ times = nullptr) {
    __shared__ R rs[3 * MAX_QS * MAX_QS + 2 * MAX_NT];
    __shared__ R sr[5 * MAX_SRC];
    const R h = (R)h_, alpha = (R)alpha_;
    for (int i = threadIdx.x; i < 3 * nq + 2 * nt; i += DIR_THREADS) rs[i] = rule[i];
    const int r = blockIdx.y;
    for (int i = threadIdx.x; i < 5 * n_src; i += DIR_THREADS) sr[i] = src[(size_t)r * n_src * 5 + i];
    __syncthreads();
    size_t idx = (size_t)blockIdx.x * DIR_THREADS + threadIdx.x;  // (k, j)
    if (idx >= (size_t)n_steps * E) return;
    const int k = (int)(idx / E), j = (int)(idx % E);
    const double *gj = geo + (size_t)j * GEO_STRIDE;
    const R *tx = rs + 3 * nq, *tw = tx + nt;
    const R nx = (R)gj[GEO_N], ny = (R)gj[GEO_N + 1], nz = (R)gj[GEO_N + 2];
    if constexpr (sizeof(R) == 4 && !NEU) {
        if (n_src == 1 && !times) {
            const R *S = sr;
            const OneSourceGeom G = one_source_geom(gj, S);
            float acc1 = 0.f;
            for (int b = 0; b < nt; ++b) {
                const float tau = (k + tx[b]) * h - S[3];
                if (tau <= 0.f) continue;
                const float q4 = 4.f * alpha * tau, c1 = -1.44269504f / q4;
                const float sq = 3.14159265f * q4;
                float sa = 0.f;
                for (int a = 0; a < nq; ++a) {
                    const float s1 = rs[3 * a], s2 = rs[3 * a + 1];
                    float rr = 0.f;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float d = fmaf(s2, G.e2[c], fmaf(s1, G.e1[c], G.p[c]));
                        rr = fmaf(d, d, rr);
                    }
                    sa = fmaf(rs[3 * a + 2], ex2_approx(rr * c1), sa);
                }
                acc1 = fmaf(tw[b] * S[4] * rsqrtf(sq * sq * sq), sa, acc1);
            }
            g[(size_t)r * n_steps * E + idx] = 2.0 * (double)acc1;
            return;
        }
    }
    R acc = 0;
    for (int a = 0; a < nq; ++a) {
        R s1 = rs[3 * a], s2 = rs[3 * a + 1], wa = rs[3 * a + 2];
        R x[3];
        for (int c = 0; c < 3; ++c)
            x[c] = (R)(gj[c] + (double)s1 * (gj[3 + c] - gj[c]) + (double)s2 * (gj[6 + c] - gj[3 + c]));
        R inner = 0;
        for (int b = 0; b < nt; ++b) {
            R t = times ? (R)(times[k] + (double)tx[b] * (times[k + 1] - times[k])) : (k + tx[b]) * h, gv = 0;
            for (int s = 0; s < n_src; ++s) {
                const R *S = sr + 5 * s;
                R d0 = x[0] - S[0], d1 = x[1] - S[1], d2 = x[2] - S[2];
                if (NEU) {
                    const R tau = t - S[3];
                    if (tau <= (R)0) continue;
                    const R dn = d0 * nx + d1 * ny + d2 * nz;
                    gv -= S[4] * heat<R>(d0 * d0 + d1 * d1 + d2 * d2, tau, alpha) * dn / ((R)2 * tau);
                } else {
                    gv = fma(S[4], heat<R>(d0 * d0 + d1 * d1 + d2 * d2, t - S[3], alpha), gv);
                }
            }
            inner = fma(tw[b], gv, inner);
        }
        acc = fma(wa, inner, acc);
    }
    g[(size_t)r * n_steps * E + idx] = 2.0 * (double)acc;
}

// Out-partials of sum (g - u_h)^2 and sum g^2 over Sigma_h for piecewise-linear
// u_h (u_h = sum_v lambda_v u1_{k, node v} on step k) and the Dirichlet datum g.
template <class R>
__global__ void __launch_bounds__(DIR_THREADS)
k_error_p1(const double *__restrict__ geo, const int32_t *__restrict__ tris, int E, int N,
           const double *__restrict__ rule, int nq, int nt, const double *__restrict__ src,
           int n_src, int nrhs, int n_steps, double h_, double alpha_,
           const double *__restrict__ u1, double *__restrict__ part) {
    __shared__ R rs[3 * MAX_QS * MAX_QS + 2 * MAX_NT];
    __shared__ R sr[5 * MAX_SRC];
    const R h = (R)h_, alpha = (R)alpha_;
    __shared__ double red[2][DIR_THREADS / 32];
    for (int i = threadIdx.x; i < 3 * nq + 2 * nt; i += DIR_THREADS) rs[i] = rule[i];
    const int r = blockIdx.y;
    for (int i = threadIdx.x; i < 5 * n_src; i += DIR_THREADS) sr[i] = src[(size_t)r * n_src * 5 + i];
    __syncthreads();
    size_t idx = (size_t)blockIdx.x * DIR_THREADS + threadIdx.x;
    double e2 = 0.0, r2 = 0.0;
    if (idx < (size_t)n_steps * E) {
        const int k = (int)(idx / E), j = (int)(idx % E);
        const double *gj = geo + (size_t)j * GEO_STRIDE;
        const R *tx = rs + 3 * nq, *tw = tx + nt;
        const double *uk = u1 + ((size_t)r * n_steps + k) * N;
        const R u0 = (R)uk[tris[3 * j]], u1v = (R)uk[tris[3 * j + 1]], u2 = (R)uk[tris[3 * j + 2]];
        R e2r = 0, r2r = 0;
        for (int a = 0; a < nq; ++a) {
            R s1 = rs[3 * a], s2 = rs[3 * a + 1], wa = rs[3 * a + 2];
            R x[3];
            for (int c = 0; c < 3; ++c)
                x[c] = (R)(gj[c] + (double)s1 * (gj[3 + c] - gj[c]) + (double)s2 * (gj[6 + c] - gj[3 + c]));
            const R uh = (1 - s1) * u0 + (s1 - s2) * u1v + s2 * u2;
            R ie = 0, ir = 0;
            for (int b = 0; b < nt; ++b) {
                R t = (k + tx[b]) * h, gv = 0;
                for (int s = 0; s < n_src; ++s) {
                    const R *S = sr + 5 * s;
                    R d0 = x[0] - S[0], d1 = x[1] - S[1], d2 = x[2] - S[2];
                    gv = fma(S[4], heat<R>(d0 * d0 + d1 * d1 + d2 * d2, t - S[3], alpha), gv);
                }
                ie = fma(tw[b], (gv - uh) * (gv - uh), ie);
                ir = fma(tw[b], gv * gv, ir);
            }
            e2r = fma(wa, ie, e2r);
            r2r = fma(wa, ir, r2r);
        }
        double f = 2.0 * gj[GEO_AREA] * h_;
        e2 = (double)e2r * f;
        r2 = (double)r2r * f;
    }
    for (int o = 16; o > 0; o >>= 1) {
        e2 += __shfl_xor_sync(0xffffffffu, e2, o);
        r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = e2;
        red[1][threadIdx.x >> 5] = r2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double se = 0.0, sr2 = 0.0;
        for (int w = 0; w < DIR_THREADS / 32; ++w) {
            se += red[0][w];
            sr2 += red[1][w];
        }
        size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        part[2 * b] = se;
        part[2 * b + 1] = sr2;
    }
}

// f_{r,k,i} = (h/2) sum_{l around i} Delta_l / 3 h_{r,k,l} - f_{r,k,i}: the
// transposed p0 x p1 mass minus the product already in f, one thread per
// (r, k, l) with atomics after negating f (k_negate).
__global__ void k_negate(double *__restrict__ f, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) f[i] = -f[i];
}
__global__ void k_add_mass_p1t(const double *__restrict__ geo, const int32_t *__restrict__ tris,
                               int E, int N, size_t total, double h, const double *__restrict__ hd,
                               double *__restrict__ f) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // (r, k, l)
    if (idx >= total) return;
    const int l = (int)(idx % E);
    double *fk = f + (idx / E) * N;
    const double v = 0.5 * h * geo[(size_t)l * GEO_STRIDE + GEO_AREA] / 3.0 * hd[idx];
    atomicAdd(fk + tris[3 * l], v);
    atomicAdd(fk + tris[3 * l + 1], v);
    atomicAdd(fk + tris[3 * l + 2], v);
}

// out-partials of sum (w - w_h)^2 and sum w^2 over Sigma_h (Sec. 6.1), with
// w = alpha du/dn_x = -sum_s weight_s G (x - y_s).n_x / (2 (t - t0_s))
template <class R>
__global__ void __launch_bounds__(DIR_THREADS)
k_error(const double *__restrict__ geo, int E, const double *__restrict__ rule, int nq, int nt,
        const double *__restrict__ src, int n_src, int nrhs, int n_steps, double h_, double alpha_,
        const double *__restrict__ wh, double *__restrict__ part,
        const double *__restrict__ times = nullptr) {
    __shared__ R rs[3 * MAX_QS * MAX_QS + 2 * MAX_NT];
    __shared__ R sr[5 * MAX_SRC];
    const R h = (R)h_, alpha = (R)alpha_;
    __shared__ double red[2][DIR_THREADS / 32];
    for (int i = threadIdx.x; i < 3 * nq + 2 * nt; i += DIR_THREADS) rs[i] = rule[i];
    const int r = blockIdx.y;
    for (int i = threadIdx.x; i < 5 * n_src; i += DIR_THREADS) sr[i] = src[(size_t)r * n_src * 5 + i];
    __syncthreads();
    size_t idx = (size_t)blockIdx.x * DIR_THREADS + threadIdx.x;
    double e2 = 0.0, r2 = 0.0;
    if (idx < (size_t)n_steps * E) {
        const int k = (int)(idx / E), j = (int)(idx % E);
        const double *gj = geo + (size_t)j * GEO_STRIDE;
        const R *tx = rs + 3 * nq, *tw = tx + nt;
        const R whv = (R)wh[(size_t)r * n_steps * E + idx];
        const R nx = (R)gj[GEO_N], ny = (R)gj[GEO_N + 1], nz = (R)gj[GEO_N + 2];
        R e2r = 0, r2r = 0;
        bool done = false;
        if constexpr (sizeof(R) == 4) {
            if (n_src == 1 && !times) {
                const R *S = sr;
                const OneSourceGeom G = one_source_geom(gj, S);
                // (x - y*) . n = p.n + s1 e1.n + s2 e2.n
                const float pn = G.p[0] * nx + G.p[1] * ny + G.p[2] * nz;
                const float e1n = G.e1[0] * nx + G.e1[1] * ny + G.e1[2] * nz;
                const float e2n = G.e2[0] * nx + G.e2[1] * ny + G.e2[2] * nz;
                for (int b = 0; b < nt; ++b) {
                    const float tau = (k + tx[b]) * h - S[3];
                    const float q4 = 4.f * alpha * tau, c1 = -1.44269504f / q4;
                    const float sq = 3.14159265f * q4;
                    // w = -weight G(r, tau) (r . n) / (2 tau); zero for tau <= 0
                    const float cb = tau > 0.f ? -S[4] * rsqrtf(sq * sq * sq) / (2.f * tau) : 0.f;
                    float ie = 0.f, ir = 0.f;
                    for (int a = 0; a < nq; ++a) {
                        const float s1 = rs[3 * a], s2 = rs[3 * a + 1], wa = rs[3 * a + 2];
                        float rr = 0.f;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const float d = fmaf(s2, G.e2[c], fmaf(s1, G.e1[c], G.p[c]));
                            rr = fmaf(d, d, rr);
                        }
                        const float dn = fmaf(s2, e2n, fmaf(s1, e1n, pn));
                        const float wv = tau > 0.f ? cb * ex2_approx(rr * c1) * dn : 0.f;
                        ie = fmaf(wa, (wv - whv) * (wv - whv), ie);
                        ir = fmaf(wa, wv * wv, ir);
                    }
                    e2r = fmaf(tw[b], ie, e2r);
                    r2r = fmaf(tw[b], ir, r2r);
                }
                done = true;
            }
        }
        for (int a = 0; a < nq && !done; ++a) {
            R s1 = rs[3 * a], s2 = rs[3 * a + 1], wa = rs[3 * a + 2];
            R x[3];
            for (int c = 0; c < 3; ++c)
                x[c] = (R)(gj[c] + (double)s1 * (gj[3 + c] - gj[c]) + (double)s2 * (gj[6 + c] - gj[3 + c]));
            R ie = 0, ir = 0;
            for (int b = 0; b < nt; ++b) {
                R t = times ? (R)(times[k] + (double)tx[b] * (times[k + 1] - times[k])) : (k + tx[b]) * h, wv = 0;
                for (int s = 0; s < n_src; ++s) {
                    const R *S = sr + 5 * s;
                    R tau = t - S[3];
                    if (tau <= (R)0) continue;
                    R d0 = x[0] - S[0], d1 = x[1] - S[1], d2 = x[2] - S[2];
                    R dn = d0 * nx + d1 * ny + d2 * nz;
                    wv -= S[4] * heat<R>(d0 * d0 + d1 * d1 + d2 * d2, tau, alpha) * dn / ((R)2 * tau);
                }
                ie = fma(tw[b], (wv - whv) * (wv - whv), ie);
                ir = fma(tw[b], wv * wv, ir);
            }
            e2r = fma(wa, ie, e2r);
            r2r = fma(wa, ir, r2r);
        }
        double f = 2.0 * gj[GEO_AREA] * (times ? times[k + 1] - times[k] : h_);
        e2 = (double)e2r * f;
        r2 = (double)r2r * f;
    }
    for (int o = 16; o > 0; o >>= 1) {
        e2 += __shfl_xor_sync(0xffffffffu, e2, o);
        r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = e2;
        red[1][threadIdx.x >> 5] = r2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double se = 0.0, sr2 = 0.0;
        for (int w = 0; w < DIR_THREADS / 32; ++w) {
            se += red[0][w];
            sr2 += red[1][w];
        }
        size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        part[2 * b] = se;
        part[2 * b + 1] = sr2;
    }
}

__global__ void k_sum_pairs(const double *__restrict__ part, size_t n, double *__restrict__ out) {
    __shared__ double red[2][32];
    double a = 0.0, b = 0.0;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a;
        red[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            sa += red[0][w];
            sb += red[1][w];
        }
        out[0] = sa;
        out[1] = sb;
    }
}

// f += (h/2) Delta_l g
__global__ void k_add_mass(const double *__restrict__ geo, int E, size_t total, double h,
                           const double *__restrict__ g, double *__restrict__ f) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int l = (int)(idx % E);
    f[idx] = fma(0.5 * h * geo[(size_t)l * GEO_STRIDE + GEO_AREA], g[idx], f[idx]);
}

static stb_status check_rule_args(int nrhs, int n_src, int q, int nt) {
    if (nrhs < 1 || nrhs > 65535 || n_src < 1 || n_src > MAX_SRC || q < 1 || q > MAX_QS ||
        nt < 1 || nt > MAX_NT)
        return fail(STB_ERR_INVALID_ARG,
                    "need 1 <= nrhs <= 65535, 1 <= n_src <= %d, 1 <= q_space <= %d, 1 <= n_time <= %d",
                    MAX_SRC, MAX_QS, MAX_NT);
    return STB_OK;
}

// Rule tables per (q, n_time) in page-locked host memory, built once and
// kept for the life of the process, so that the copy below is a plain
// asynchronous copy (and can be captured into a CUDA graph once the first,
// uncaptured call has built the table).
static stb_status pinned_rules(int q, int nt, const double **out, size_t *count) {
    static std::mutex mu;
    static std::map<std::pair<int, int>, std::pair<double *, size_t>> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto f = cache.find({q, nt});
    if (f == cache.end()) {
        std::vector<double> host;
        host_rules(q, nt, host);
        double *pinned = nullptr;
        STB_CUDA(cudaMallocHost(&pinned, host.size() * sizeof(double)));
        std::copy(host.begin(), host.end(), pinned);
        f = cache.emplace(std::make_pair(q, nt), std::make_pair(pinned, host.size())).first;
    }
    *out = f->second.first;
    *count = f->second.second;
    return STB_OK;
}

static stb_status upload_rules_sources(const DirLayout &L, int q, int nt, const double *sources,
                                       int nrhs, int n_src, cudaStream_t s) {
    const double *rules;
    size_t count;
    stb_status st = pinned_rules(q, nt, &rules, &count);
    if (st) return st;
    STB_CUDA(cudaMemcpyAsync(L.rule, rules, count * sizeof(double), cudaMemcpyHostToDevice, s));
    STB_CUDA(cudaMemcpyAsync(L.src, sources, sizeof(double) * 5 * (size_t)nrhs * n_src,
                             cudaMemcpyHostToDevice, s));
    return STB_OK;
}

// ------------------------------------ piecewise-linear data (Sec. 3.4) ---
// Nodal moments b_{r,k,i} = h^{-1} int_{t_k}^{t_{k+1}} int_Gamma g_r phi_i of
// the hat functions phi_i: per element (r, k, j) the three vertex moments
// 2 Delta_j sum_a w_a lambda_v(a) (time mean of g_r at x_a), added to the
// nodes of triangle j (atomics: b starts at zero).
template <class R>
__global__ void __launch_bounds__(DIR_THREADS)
k_project_p1(const double *__restrict__ geo, const int32_t *__restrict__ tris, int E, int N,
             const double *__restrict__ rule, int nq, int nt, const double *__restrict__ src,
             int n_src, int n_steps, double h_, double alpha_, double *__restrict__ b) {
    __shared__ R rs[3 * MAX_QS * MAX_QS + 2 * MAX_NT];
    __shared__ R sr[5 * MAX_SRC];
    const R h = (R)h_, alpha = (R)alpha_;
    for (int i = threadIdx.x; i < 3 * nq + 2 * nt; i += DIR_THREADS) rs[i] = rule[i];
    const int r = blockIdx.y;
    for (int i = threadIdx.x; i < 5 * n_src; i += DIR_THREADS) sr[i] = src[(size_t)r * n_src * 5 + i];
    __syncthreads();
    size_t idx = (size_t)blockIdx.x * DIR_THREADS + threadIdx.x;  // (k, j)
    if (idx >= (size_t)n_steps * E) return;
    const int k = (int)(idx / E), j = (int)(idx % E);
    const double *gj = geo + (size_t)j * GEO_STRIDE;
    const R *tx = rs + 3 * nq, *tw = tx + nt;
    R acc[3] = {0, 0, 0};
    for (int a = 0; a < nq; ++a) {
        R s1 = rs[3 * a], s2 = rs[3 * a + 1], wa = rs[3 * a + 2];
        R x[3];
        for (int c = 0; c < 3; ++c)
            x[c] = (R)(gj[c] + (double)s1 * (gj[3 + c] - gj[c]) + (double)s2 * (gj[6 + c] - gj[3 + c]));
        R inner = 0;
        for (int q = 0; q < nt; ++q) {
            R t = (k + tx[q]) * h, gv = 0;
            for (int si = 0; si < n_src; ++si) {
                const R *S = sr + 5 * si;
                R d0 = x[0] - S[0], d1 = x[1] - S[1], d2 = x[2] - S[2];
                gv = fma(S[4], heat<R>(d0 * d0 + d1 * d1 + d2 * d2, t - S[3], alpha), gv);
            }
            inner = fma(tw[q], gv, inner);
        }
        const R wi = wa * inner;
        acc[0] = fma(1 - s1, wi, acc[0]);
        acc[1] = fma(s1 - s2, wi, acc[1]);
        acc[2] = fma(s2, wi, acc[2]);
    }
    double *bk = b + ((size_t)r * n_steps + k) * N;
    const double area2 = 2.0 * gj[GEO_AREA];
#pragma unroll
    for (int v = 0; v < 3; ++v) atomicAdd(bk + tris[3 * j + v], area2 * (double)acc[v]);
}

// Mass matrix of the hat functions: M1[i][i'] += Delta_j / 12 (1 + [i = i'])
// over the vertices i, i' of every triangle j (M1 starts at zero).
__global__ void k_mass_p1(const double *__restrict__ geo, const int32_t *__restrict__ tris, int E,
                          int N, double *__restrict__ M) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= E) return;
    const double m = geo[(size_t)j * GEO_STRIDE + GEO_AREA] / 12.0;
    const int t[3] = {tris[3 * j], tris[3 * j + 1], tris[3 * j + 2]};
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) atomicAdd(M + (size_t)t[a] * N + t[c], a == c ? 2.0 * m : m);
}

// f_{r,k,l} += (h/2) (Delta_l / 3) sum over the vertices i of l of g1_{r,k,i}
// (the p0 x p1 mass matrix: int_{gamma_l} phi_i = Delta_l / 3)
__global__ void k_add_mass_p1(const double *__restrict__ geo, const int32_t *__restrict__ tris,
                              int E, int N, size_t total, double h, const double *__restrict__ g1,
                              double *__restrict__ f) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int l = (int)(idx % E);
    const double *gk = g1 + (idx / E) * N;
    const double m = gk[tris[3 * l]] + gk[tris[3 * l + 1]] + gk[tris[3 * l + 2]];
    f[idx] = fma(0.5 * h * geo[(size_t)l * GEO_STRIDE + GEO_AREA] / 3.0, m, f[idx]);
}

// Every node must belong to a triangle, else M1 is singular.
static stb_status check_nodes_used(const Mesh &m) {
    std::vector<char> used(m.n_nodes, 0);
    for (int32_t t : m.tris) used[t] = 1;
    for (int64_t i = 0; i < m.n_nodes; ++i)
        if (!used[i]) return fail(STB_ERR_INVALID_ARG, "node %lld belongs to no triangle", (long long)i);
    if (m.n_nodes > 65535) return fail(STB_ERR_INVALID_ARG, "n_nodes must be <= 65535");
    return STB_OK;
}

// Workspace of the p1 projection: rules, sources and geometry, the mass
// matrix, the moments, the scratch of its inverse.
struct P1Layout {
    DirLayout d;
    double *M, *b;
    void *inv;
    size_t inv_bytes, bytes;
};

static P1Layout p1_layout(const Mesh &m, int n_steps, int nrhs, int n_src, int q, int nt, void *ws,
                          size_t cap) {
    P1Layout P{};
    P.d = dir_layout(m, nrhs, n_src, q, nt, ws, cap, 0);
    Carve c(ws, cap);
    c.off = P.d.bytes;
    const size_t N = (size_t)m.n_nodes;
    P.M = c.take<double>(N * N);
    P.b = c.take<double>((size_t)nrhs * n_steps * N);
    P.inv_bytes = spd_inverse_bytes((int64_t)N);
    P.inv = c.take<char>(P.inv_bytes);
    P.bytes = c.off;
    return P;
}

}  // namespace stb

using namespace stb;

extern "C" stb_status stb_project_workspace_size(const stb_mesh *mesh, int32_t nrhs, int32_t n_src,
                                                 int32_t q, int32_t nt, size_t *bytes) {
    if (!mesh || !bytes) return fail(STB_ERR_INVALID_ARG, "mesh and bytes must be given");
    stb_status st = check_rule_args(nrhs, n_src, q, nt);
    if (st) return st;
    *bytes = align256(dir_layout(mesh->m, nrhs, n_src, q, nt, nullptr, 0, 0).bytes);
    return STB_OK;
}

extern "C" stb_status stb_project_dirichlet(const stb_mesh *mesh, const stb_params *p,
                                            const double *sources, int32_t nrhs, int32_t n_src,
                                            int32_t q, int32_t nt, double *g, void *ws,
                                            size_t ws_bytes, stb_stream stream) {
    if (!mesh || !p || !sources || !g) return fail(STB_ERR_INVALID_ARG, "null argument");
    if (!(p->alpha > 0) || !(p->T > 0) || p->n_steps < 1)
        return fail(STB_ERR_INVALID_ARG, "alpha, T and n_steps must be positive");
    stb_status st = check_rule_args(nrhs, n_src, q, nt);
    if (st) return st;
    const Mesh &m = mesh->m;
    DirLayout L = dir_layout(m, nrhs, n_src, q, nt, ws, ws_bytes, 0);
    if ((st = check_workspace(ws, ws_bytes, L.bytes))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    if ((st = upload_rules_sources(L, q, nt, sources, nrhs, n_src, s))) return st;
    if ((st = launch_geometry(m, L.geo, s))) return st;
    size_t n = (size_t)p->n_steps * m.n_tris;
    dim3 grid((unsigned)((n + DIR_THREADS - 1) / DIR_THREADS), (unsigned)nrhs);
    count_launch(s);
    if (p->precision == STB_PREC_MIXED)
        k_project<float><<<grid, DIR_THREADS, 0, s>>>(L.geo, (int)m.n_tris, L.rule, q * q, nt, L.src,
                                                      n_src, nrhs, p->n_steps, p->T / p->n_steps,
                                                      p->alpha, g);
    else
        k_project<double><<<grid, DIR_THREADS, 0, s>>>(L.geo, (int)m.n_tris, L.rule, q * q, nt, L.src,
                                                       n_src, nrhs, p->n_steps, p->T / p->n_steps,
                                                       p->alpha, g);
    return check_launch("k_project");
}

extern "C" stb_status stb_rhs_workspace_size(const stb_mesh *mesh, const stb_params *p, int32_t nrhs,
                                             size_t *bytes) {
    if (!mesh || !p || !bytes || nrhs < 1 || p->n_steps < 1)
        return fail(STB_ERR_INVALID_ARG, "invalid argument");
    Carve c(nullptr, 0);
    c.take<double>((size_t)mesh->m.n_tris * GEO_STRIDE);
    c.take<char>(p->precision == STB_PREC_MIXED
                     ? toeplitz_split_bytes(mesh->m.n_tris, p->n_steps, nrhs)
                     : toeplitz_partial_bytes(mesh->m.n_tris, p->n_steps, nrhs));
    *bytes = align256(c.off);
    return STB_OK;
}

extern "C" stb_status stb_dirichlet_rhs(const stb_mesh *mesh, const stb_params *p, const void *K,
                                        const double *g, int32_t nrhs, double *f, void *ws,
                                        size_t ws_bytes, stb_stream stream) {
    if (!mesh || !p || !K || !g || !f) return fail(STB_ERR_INVALID_ARG, "null argument");
    if (p->storage != STB_STORE_F64 && p->storage != STB_STORE_F32)
        return fail(STB_ERR_INVALID_ARG, "bad storage");
    size_t need;
    stb_status st = stb_rhs_workspace_size(mesh, p, nrhs, &need);
    if (st) return st;
    if ((st = check_workspace(ws, ws_bytes, need))) return st;
    const Mesh &m = mesh->m;
    const bool mixed = p->precision == STB_PREC_MIXED;
    if (mixed && p->storage != STB_STORE_F32)
        return fail(STB_ERR_INVALID_ARG, "mixed precision needs STB_STORE_F32 blocks");
    Carve c(ws, ws_bytes);
    double *geo = c.take<double>((size_t)m.n_tris * GEO_STRIDE);
    void *part = c.take<char>(mixed ? toeplitz_split_bytes(m.n_tris, p->n_steps, nrhs)
                                    : toeplitz_partial_bytes(m.n_tris, p->n_steps, nrhs));
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    if ((st = launch_geometry(m, geo, s))) return st;
    if (mixed)  // K g on the tensor cores with split operands
        st = toeplitz_split((const float *)K, m.n_tris, p->n_steps, nrhs, g, DF_AXPBY, nullptr, 0.0,
                            f, part, status_word(ws), s);
    else
        st = toeplitz_fp64(K, p->storage, m.n_tris, p->n_steps, nrhs, g, 0.0, f, (double *)part, s);
    if (st) return st;
    size_t total = (size_t)nrhs * p->n_steps * m.n_tris;
    count_launch(s);
    k_add_mass<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(geo, (int)m.n_tris, total,
                                                                p->T / p->n_steps, g, f);
    return check_launch("k_add_mass");
}

static size_t error_blocks(const Mesh &m, int n_steps, int nrhs) {
    size_t n = (size_t)n_steps * m.n_tris;
    return ((n + DIR_THREADS - 1) / DIR_THREADS) * (size_t)nrhs;
}

extern "C" stb_status stb_error_workspace_size(const stb_mesh *mesh, const stb_params *p,
                                               int32_t nrhs, int32_t n_src, int32_t q, int32_t nt,
                                               size_t *bytes) {
    if (!mesh || !p || !bytes || p->n_steps < 1) return fail(STB_ERR_INVALID_ARG, "invalid argument");
    stb_status st = check_rule_args(nrhs, n_src, q, nt);
    if (st) return st;
    size_t nblk = error_blocks(mesh->m, p->n_steps, nrhs);
    *bytes = align256(dir_layout(mesh->m, nrhs, n_src, q, nt, nullptr, 0, 2 * nblk).bytes);
    return STB_OK;
}

extern "C" stb_status stb_neumann_error(const stb_mesh *mesh, const stb_params *p,
                                        const double *sources, int32_t nrhs, int32_t n_src,
                                        const double *w, int32_t q, int32_t nt, double *out,
                                        void *ws, size_t ws_bytes, stb_stream stream) {
    if (!mesh || !p || !sources || !w || !out) return fail(STB_ERR_INVALID_ARG, "null argument");
    if (!(p->alpha > 0) || !(p->T > 0) || p->n_steps < 1 || p->n_steps > 4096)
        return fail(STB_ERR_INVALID_ARG, "alpha, T must be positive, 1 <= n_steps <= 4096");
    stb_status st = check_rule_args(nrhs, n_src, q, nt);
    if (st) return st;
    const Mesh &m = mesh->m;
    size_t n = (size_t)p->n_steps * m.n_tris;
    unsigned gx = (unsigned)((n + DIR_THREADS - 1) / DIR_THREADS);
    size_t nblk = error_blocks(m, p->n_steps, nrhs);
    DirLayout L = dir_layout(m, nrhs, n_src, q, nt, ws, ws_bytes, 2 * nblk);
    if ((st = check_workspace(ws, ws_bytes, L.bytes))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    if ((st = upload_rules_sources(L, q, nt, sources, nrhs, n_src, s))) return st;
    if ((st = launch_geometry(m, L.geo, s))) return st;
    count_launch(s);
    if (p->precision == STB_PREC_MIXED)
        k_error<float><<<dim3(gx, (unsigned)nrhs), DIR_THREADS, 0, s>>>(
            L.geo, (int)m.n_tris, L.rule, q * q, nt, L.src, n_src, nrhs, p->n_steps, p->T / p->n_steps,
            p->alpha, w, L.part);
    else
        k_error<double><<<dim3(gx, (unsigned)nrhs), DIR_THREADS, 0, s>>>(
            L.geo, (int)m.n_tris, L.rule, q * q, nt, L.src, n_src, nrhs, p->n_steps, p->T / p->n_steps,
            p->alpha, w, L.part);
    if ((st = check_launch("k_error"))) return st;
    count_launch(s);
    k_sum_pairs<<<1, 1024, 0, s>>>(L.part, nblk, out);
    return check_launch("k_sum_pairs");
}

// ---------------------------------------- piecewise-linear data (Sec. 3.4) ---
extern "C" stb_status stb_project_p1_workspace_size(const stb_mesh *mesh, const stb_params *p,
                                                    int32_t nrhs, int32_t n_src, int32_t q,
                                                    int32_t nt, size_t *bytes) {
    if (!mesh || !p || !bytes || p->n_steps < 1) return fail(STB_ERR_INVALID_ARG, "invalid argument");
    stb_status st = check_rule_args(nrhs, n_src, q, nt);
    if (st) return st;
    if ((st = check_nodes_used(mesh->m))) return st;
    *bytes = align256(p1_layout(mesh->m, p->n_steps, nrhs, n_src, q, nt, nullptr, 0).bytes);
    return STB_OK;
}

extern "C" stb_status stb_project_dirichlet_p1(const stb_mesh *mesh, const stb_params *p,
                                               const double *sources, int32_t nrhs, int32_t n_src,
                                               int32_t q, int32_t nt, double *g1, void *ws,
                                               size_t ws_bytes, stb_stream stream) {
    if (!mesh || !p || !sources || !g1) return fail(STB_ERR_INVALID_ARG, "null argument");
    if (!(p->alpha > 0) || !(p->T > 0) || p->n_steps < 1)
        return fail(STB_ERR_INVALID_ARG, "alpha, T and n_steps must be positive");
    size_t need;
    stb_status st = stb_project_p1_workspace_size(mesh, p, nrhs, n_src, q, nt, &need);
    if (st) return st;
    if ((st = check_workspace(ws, ws_bytes, need))) return st;
    const Mesh &m = mesh->m;
    const int E = (int)m.n_tris, N = (int)m.n_nodes;
    P1Layout P = p1_layout(m, p->n_steps, nrhs, n_src, q, nt, ws, ws_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    if ((st = upload_rules_sources(P.d, q, nt, sources, nrhs, n_src, s))) return st;
    if ((st = launch_geometry(m, P.d.geo, s))) return st;
    // mass matrix and its inverse
    STB_CUDA(cudaMemsetAsync(P.M, 0, sizeof(double) * (size_t)N * N, s));
    count_launch(s);
    k_mass_p1<<<(E + 127) / 128, 128, 0, s>>>(P.d.geo, m.d_tris, E, N, P.M);
    if ((st = check_launch("k_mass_p1"))) return st;
    double *inv = nullptr;
    if ((st = spd_inverse(P.M, N, P.inv, P.inv_bytes, status_word(ws), &inv, s))) return st;
    // moments, then g1 = M1^{-1} b for every (r, k)
    const size_t nb = (size_t)nrhs * p->n_steps * N;
    STB_CUDA(cudaMemsetAsync(P.b, 0, sizeof(double) * nb, s));
    const size_t n = (size_t)p->n_steps * E;
    dim3 grid((unsigned)((n + DIR_THREADS - 1) / DIR_THREADS), (unsigned)nrhs);
    count_launch(s);
    if (p->precision == STB_PREC_MIXED)
        k_project_p1<float><<<grid, DIR_THREADS, 0, s>>>(P.d.geo, m.d_tris, E, N, P.d.rule, q * q,
                                                         nt, P.d.src, n_src, p->n_steps,
                                                         p->T / p->n_steps, p->alpha, P.b);
    else
        k_project_p1<double><<<grid, DIR_THREADS, 0, s>>>(P.d.geo, m.d_tris, E, N, P.d.rule, q * q,
                                                          nt, P.d.src, n_src, p->n_steps,
                                                          p->T / p->n_steps, p->alpha, P.b);
    if ((st = check_launch("k_project_p1"))) return st;
    return dense_apply(inv, N, (int64_t)nrhs * p->n_steps, P.b, g1, s);
}

extern "C" stb_status stb_rhs_p1_workspace_size(const stb_mesh *mesh, const stb_params *p,
                                                int32_t nrhs, size_t *bytes) {
    if (!mesh || !p || !bytes || nrhs < 1 || p->n_steps < 1)
        return fail(STB_ERR_INVALID_ARG, "invalid argument");
    Carve c(nullptr, 0);
    c.take<double>((size_t)mesh->m.n_tris * GEO_STRIDE);
    c.take<char>(toeplitz_partial_bytes(mesh->m.n_tris, p->n_steps, nrhs));
    *bytes = align256(c.off);
    return STB_OK;
}

extern "C" stb_status stb_dirichlet_rhs_p1(const stb_mesh *mesh, const stb_params *p,
                                           const void *K1, const double *g1, int32_t nrhs,
                                           double *f, void *ws, size_t ws_bytes, stb_stream stream) {
    if (!mesh || !p || !K1 || !g1 || !f) return fail(STB_ERR_INVALID_ARG, "null argument");
    if (p->storage != STB_STORE_F64 && p->storage != STB_STORE_F32)
        return fail(STB_ERR_INVALID_ARG, "bad storage");
    size_t need;
    stb_status st = stb_rhs_p1_workspace_size(mesh, p, nrhs, &need);
    if (st) return st;
    if ((st = check_workspace(ws, ws_bytes, need))) return st;
    const Mesh &m = mesh->m;
    Carve c(ws, ws_bytes);
    double *geo = c.take<double>((size_t)m.n_tris * GEO_STRIDE);
    double *part = (double *)c.take<char>(toeplitz_partial_bytes(m.n_tris, p->n_steps, nrhs));
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    if ((st = launch_geometry(m, geo, s))) return st;
    if ((st = toeplitz_fp64_rect(K1, p->storage, m.n_tris, m.n_nodes, p->n_steps, nrhs, g1, 0.0, f,
                                 part, s)))
        return st;
    const size_t total = (size_t)nrhs * p->n_steps * m.n_tris;
    count_launch(s);
    k_add_mass_p1<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
        geo, m.d_tris, (int)m.n_tris, (int)m.n_nodes, total, p->T / p->n_steps, g1, f);
    return check_launch("k_add_mass_p1");
}

// ---------------------------------------------- Neumann problem (Sec. 3.4) ---
extern "C" stb_status stb_project_neumann(const stb_mesh *mesh, const stb_params *p,
                                          const double *sources, int32_t nrhs, int32_t n_src,
                                          int32_t q, int32_t nt, double *hd, void *ws,
                                          size_t ws_bytes, stb_stream stream) {
    if (!mesh || !p || !sources || !hd) return fail(STB_ERR_INVALID_ARG, "null argument");
    if (!(p->alpha > 0) || !(p->T > 0) || p->n_steps < 1)
        return fail(STB_ERR_INVALID_ARG, "alpha, T and n_steps must be positive");
    stb_status st = check_rule_args(nrhs, n_src, q, nt);
    if (st) return st;
    const Mesh &m = mesh->m;
    DirLayout L = dir_layout(m, nrhs, n_src, q, nt, ws, ws_bytes, 0);
    if ((st = check_workspace(ws, ws_bytes, L.bytes))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    if ((st = upload_rules_sources(L, q, nt, sources, nrhs, n_src, s))) return st;
    if ((st = launch_geometry(m, L.geo, s))) return st;
    size_t n = (size_t)p->n_steps * m.n_tris;
    dim3 grid((unsigned)((n + DIR_THREADS - 1) / DIR_THREADS), (unsigned)nrhs);
    count_launch(s);
    if (p->precision == STB_PREC_MIXED)
        k_project<float, true><<<grid, DIR_THREADS, 0, s>>>(L.geo, (int)m.n_tris, L.rule, q * q, nt,
                                                            L.src, n_src, nrhs, p->n_steps,
                                                            p->T / p->n_steps, p->alpha, hd);
    else
        k_project<double, true><<<grid, DIR_THREADS, 0, s>>>(L.geo, (int)m.n_tris, L.rule, q * q, nt,
                                                             L.src, n_src, nrhs, p->n_steps,
                                                             p->T / p->n_steps, p->alpha, hd);
    return check_launch("k_project(neumann)");
}

extern "C" stb_status stb_dirichlet_error_p1(const stb_mesh *mesh, const stb_params *p,
                                             const double *sources, int32_t nrhs, int32_t n_src,
                                             const double *u1, int32_t q, int32_t nt, double *out,
                                             void *ws, size_t ws_bytes, stb_stream stream) {
    if (!mesh || !p || !sources || !u1 || !out) return fail(STB_ERR_INVALID_ARG, "null argument");
    if (!(p->alpha > 0) || !(p->T > 0) || p->n_steps < 1)
        return fail(STB_ERR_INVALID_ARG, "alpha, T and n_steps must be positive");
    stb_status st = check_rule_args(nrhs, n_src, q, nt);
    if (st) return st;
    const Mesh &m = mesh->m;
    const size_t nblk = error_blocks(m, p->n_steps, nrhs);
    DirLayout L = dir_layout(m, nrhs, n_src, q, nt, ws, ws_bytes, 2 * nblk);
    if ((st = check_workspace(ws, ws_bytes, L.bytes))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    if ((st = upload_rules_sources(L, q, nt, sources, nrhs, n_src, s))) return st;
    if ((st = launch_geometry(m, L.geo, s))) return st;
    size_t n = (size_t)p->n_steps * m.n_tris;
    dim3 grid((unsigned)((n + DIR_THREADS - 1) / DIR_THREADS), (unsigned)nrhs);
    count_launch(s);
    if (p->precision == STB_PREC_MIXED)
        k_error_p1<float><<<grid, DIR_THREADS, 0, s>>>(L.geo, m.d_tris, (int)m.n_tris, (int)m.n_nodes,
                                                       L.rule, q * q, nt, L.src, n_src, nrhs,
                                                       p->n_steps, p->T / p->n_steps, p->alpha, u1,
                                                       L.part);
    else
        k_error_p1<double><<<grid, DIR_THREADS, 0, s>>>(L.geo, m.d_tris, (int)m.n_tris,
                                                        (int)m.n_nodes, L.rule, q * q, nt, L.src,
                                                        n_src, nrhs, p->n_steps, p->T / p->n_steps,
                                                        p->alpha, u1, L.part);
    if ((st = check_launch("k_error_p1"))) return st;
    count_launch(s);
    k_sum_pairs<<<1, 1024, 0, s>>>(L.part, nblk, out);
    return check_launch("k_sum_pairs");
}

extern "C" stb_status stb_neumann_rhs_workspace_size(const stb_mesh *mesh, const stb_params *p,
                                                     int32_t nrhs, size_t *bytes) {
    if (!mesh || !p || !bytes || nrhs < 1 || p->n_steps < 1)
        return fail(STB_ERR_INVALID_ARG, "invalid argument");
    Carve c(nullptr, 0);
    c.take<double>((size_t)mesh->m.n_tris * GEO_STRIDE);
    c.take<char>(toeplitz_partial_bytes(mesh->m.n_nodes, p->n_steps, nrhs));
    *bytes = align256(c.off);
    return STB_OK;
}

extern "C" stb_status stb_neumann_rhs(const stb_mesh *mesh, const stb_params *p, const void *K1,
                                      const double *hd, int32_t nrhs, double *f, void *ws,
                                      size_t ws_bytes, stb_stream stream) {
    if (!mesh || !p || !K1 || !hd || !f) return fail(STB_ERR_INVALID_ARG, "null argument");
    if (p->storage != STB_STORE_F64 && p->storage != STB_STORE_F32)
        return fail(STB_ERR_INVALID_ARG, "bad storage");
    size_t need;
    stb_status st = stb_neumann_rhs_workspace_size(mesh, p, nrhs, &need);
    if (st) return st;
    if ((st = check_workspace(ws, ws_bytes, need))) return st;
    const Mesh &m = mesh->m;
    Carve c(ws, ws_bytes);
    double *geo = c.take<double>((size_t)m.n_tris * GEO_STRIDE);
    double *part = (double *)c.take<char>(toeplitz_partial_bytes(m.n_nodes, p->n_steps, nrhs));
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    if ((st = launch_geometry(m, geo, s))) return st;
    if ((st = toeplitz_fp64_rect_t(K1, p->storage, m.n_tris, m.n_nodes, p->n_steps, nrhs, hd, 0.0,
                                   f, part, s)))
        return st;
    const size_t nf = (size_t)nrhs * p->n_steps * m.n_nodes;
    count_launch(s);
    k_negate<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(f, nf);
    if ((st = check_launch("k_negate"))) return st;
    const size_t total = (size_t)nrhs * p->n_steps * m.n_tris;
    count_launch(s);
    k_add_mass_p1t<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
        geo, m.d_tris, (int)m.n_tris, (int)m.n_nodes, total, p->T / p->n_steps, hd, f);
    return check_launch("k_add_mass_p1t");
}

// ------------------------------------------ non-uniform time grids (Sec. 7) ---
static stb_status nu_times_check(const stb_params *p, const double *times) {
    if (!p || !times) return fail(STB_ERR_INVALID_ARG, "params and times must be given");
    if (p->n_steps < 1 || times[0] != 0.0) return fail(STB_ERR_INVALID_ARG, "need n_steps >= 1, times[0] = 0");
    for (int k = 0; k < p->n_steps; ++k)
        if (!(times[k + 1] > times[k])) return fail(STB_ERR_INVALID_ARG, "times must increase strictly");
    return STB_OK;
}

// f^k += (h_k / 2) Delta_l g^k
__global__ void k_add_mass_nu(const double *__restrict__ geo, int E, int n_steps, size_t total,
                              const double *__restrict__ times, const double *__restrict__ g,
                              double *__restrict__ f) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int l = (int)(idx % E), k = (int)((idx / E) % n_steps);
    const double h = times[k + 1] - times[k];
    f[idx] = fma(0.5 * h * geo[(size_t)l * GEO_STRIDE + GEO_AREA], g[idx], f[idx]);
}

extern "C" stb_status stb_project_nu_workspace_size(const stb_mesh *mesh, const stb_params *p,
                                                    int32_t nrhs, int32_t n_src, int32_t q,
                                                    int32_t nt, size_t *bytes) {
    if (!mesh || !p || !bytes) return fail(STB_ERR_INVALID_ARG, "invalid argument");
    stb_status st = check_rule_args(nrhs, n_src, q, nt);
    if (st) return st;
    const size_t nblk = error_blocks(mesh->m, p->n_steps, nrhs);
    *bytes = align256(dir_layout(mesh->m, nrhs, n_src, q, nt, nullptr, 0, 2 * nblk).bytes) +
             align256(sizeof(double) * (p->n_steps + 1));
    return STB_OK;
}

// project (mode 0) or error (mode 1) on a non-uniform grid
static stb_status nu_data(int mode, const stb_mesh *mesh, const stb_params *p, const double *times,
                          const double *sources, int32_t nrhs, int32_t n_src, int32_t q,
                          int32_t nt, const double *w, double *out, void *ws, size_t ws_bytes,
                          cudaStream_t s) {
    if (!mesh || !sources || !out || (mode == 1 && !w)) return fail(STB_ERR_INVALID_ARG, "null argument");
    stb_status st = nu_times_check(p, times);
    if (st) return st;
    if (!(p->alpha > 0)) return fail(STB_ERR_INVALID_ARG, "alpha must be positive");
    size_t need;
    if ((st = stb_project_nu_workspace_size(mesh, p, nrhs, n_src, q, nt, &need))) return st;
    if ((st = check_workspace(ws, ws_bytes, need))) return st;
    const Mesh &m = mesh->m;
    const size_t nblk = error_blocks(m, p->n_steps, nrhs);
    DirLayout L = dir_layout(m, nrhs, n_src, q, nt, ws, ws_bytes, 2 * nblk);
    double *d_times = reinterpret_cast<double *>(static_cast<char *>(ws) + align256(L.bytes));
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    if ((st = upload_rules_sources(L, q, nt, sources, nrhs, n_src, s))) return st;
    STB_CUDA(cudaMemcpyAsync(d_times, times, sizeof(double) * (p->n_steps + 1),
                             cudaMemcpyHostToDevice, s));
    if ((st = launch_geometry(m, L.geo, s))) return st;
    const size_t n = (size_t)p->n_steps * m.n_tris;
    dim3 grid((unsigned)((n + DIR_THREADS - 1) / DIR_THREADS), (unsigned)nrhs);
    count_launch(s);
    if (mode == 0) {
        k_project<double><<<grid, DIR_THREADS, 0, s>>>(L.geo, (int)m.n_tris, L.rule, q * q, nt,
                                                       L.src, n_src, nrhs, p->n_steps, 0.0,
                                                       p->alpha, out, d_times);
        return check_launch("k_project(non-uniform)");
    }
    k_error<double><<<grid, DIR_THREADS, 0, s>>>(L.geo, (int)m.n_tris, L.rule, q * q, nt, L.src,
                                                 n_src, nrhs, p->n_steps, 0.0, p->alpha, w, L.part,
                                                 d_times);
    if ((st = check_launch("k_error(non-uniform)"))) return st;
    count_launch(s);
    k_sum_pairs<<<1, 1024, 0, s>>>(L.part, nblk, out);
    return check_launch("k_sum_pairs");
}

extern "C" stb_status stb_project_dirichlet_nu(const stb_mesh *mesh, const stb_params *p,
                                               const double *times, const double *sources,
                                               int32_t nrhs, int32_t n_src, int32_t q, int32_t nt,
                                               double *g, void *ws, size_t ws_bytes,
                                               stb_stream stream) {
    return nu_data(0, mesh, p, times, sources, nrhs, n_src, q, nt, nullptr, g, ws, ws_bytes,
                   (cudaStream_t)stream);
}

extern "C" stb_status stb_neumann_error_nu(const stb_mesh *mesh, const stb_params *p,
                                           const double *times, const double *sources,
                                           int32_t nrhs, int32_t n_src, const double *w, int32_t q,
                                           int32_t nt, double *out, void *ws, size_t ws_bytes,
                                           stb_stream stream) {
    return nu_data(1, mesh, p, times, sources, nrhs, n_src, q, nt, w, out, ws, ws_bytes,
                   (cudaStream_t)stream);
}

extern "C" stb_status stb_dirichlet_rhs_nu_workspace_size(const stb_mesh *mesh,
                                                          const stb_params *p, size_t *bytes) {
    if (!mesh || !p || !bytes || p->n_steps < 1) return fail(STB_ERR_INVALID_ARG, "invalid argument");
    *bytes = align256(256 + align256(sizeof(double) * mesh->m.n_tris * GEO_STRIDE) +
                      align256(sizeof(double) * (p->n_steps + 1)));
    return STB_OK;
}

extern "C" stb_status stb_dirichlet_rhs_nu(const stb_mesh *mesh, const stb_params *p,
                                           const double *times, const double *K, const double *g,
                                           int32_t nrhs, double *f, void *ws, size_t ws_bytes,
                                           stb_stream stream) {
    if (!mesh || !K || !g || !f || nrhs < 1) return fail(STB_ERR_INVALID_ARG, "null argument");
    stb_status st = nu_times_check(p, times);
    if (st) return st;
    size_t need;
    if ((st = stb_dirichlet_rhs_nu_workspace_size(mesh, p, &need))) return st;
    if ((st = check_workspace(ws, ws_bytes, need))) return st;
    const Mesh &m = mesh->m;
    Carve c(ws, ws_bytes);
    double *geo = c.take<double>((size_t)m.n_tris * GEO_STRIDE);
    double *d_times = c.take<double>(p->n_steps + 1);
    cudaStream_t s = (cudaStream_t)stream;
    STB_CUDA(cudaMemsetAsync(ws, 0, 256, s));
    STB_CUDA(cudaMemcpyAsync(d_times, times, sizeof(double) * (p->n_steps + 1),
                             cudaMemcpyHostToDevice, s));
    if ((st = launch_geometry(m, geo, s))) return st;
    if ((st = matvec_nu(K, m.n_tris, p->n_steps, nrhs, g, f, s))) return st;
    const size_t total = (size_t)nrhs * p->n_steps * m.n_tris;
    count_launch(s);
    k_add_mass_nu<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(geo, (int)m.n_tris, p->n_steps,
                                                                  total, d_times, g, f);
    return check_launch("k_add_mass_nu");
}

