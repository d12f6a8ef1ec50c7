// stb_host.cpp -- host side of the library: error reporting, mesh validation
// and upload, quadrature tables (generated at run time), workspace checks.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <unordered_set>

#include "stb_internal.h"

namespace stb {

static thread_local std::string t_last_error;
std::atomic<int64_t> g_launches{0};

stb_status fail(stb_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return code;
}

stb_status cuda_fail(cudaError_t err, const char *what) {
    return fail(STB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(err));
}

// ---- tracing: events around launches (see stb_trace_* in stbem.h) ----------
struct TraceRec {
    const char *name;
    cudaEvent_t a, b;
};
static std::atomic<bool> g_trace_on{false};
static std::mutex g_trace_mu;
static std::vector<TraceRec> g_trace_pending;
static std::vector<cudaEvent_t> g_trace_pool;
static std::map<std::string, std::pair<int64_t, double>> g_trace_acc;
static thread_local int t_open = -1;
static thread_local cudaStream_t t_open_stream = nullptr;

static cudaEvent_t trace_event() {
    if (!g_trace_pool.empty()) {
        cudaEvent_t e = g_trace_pool.back();
        g_trace_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void count_launch(cudaStream_t s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    t_open = -1;
    if (!g_trace_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_trace_mu);
    TraceRec r{nullptr, trace_event(), trace_event()};
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, s);
    g_trace_pending.push_back(r);
    t_open = (int)g_trace_pending.size() - 1;
    t_open_stream = s;
}

stb_status check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (t_open >= 0) {
        std::lock_guard<std::mutex> lk(g_trace_mu);
        if (t_open < (int)g_trace_pending.size()) {
            g_trace_pending[t_open].name = what;
            cudaEventRecord(g_trace_pending[t_open].b, t_open_stream);
        }
        t_open = -1;
    }
    if (e != cudaSuccess) return cuda_fail(e, what);
    return STB_OK;
}

static stb_status trace_drain() {
    std::lock_guard<std::mutex> lk(g_trace_mu);
    for (auto &r : g_trace_pending) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize(trace)");
        float ms = 0.f;
        if (r.name && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            auto &acc = g_trace_acc[r.name];
            acc.first += 1;
            acc.second += ms;
        }
        g_trace_pool.push_back(r.a);
        g_trace_pool.push_back(r.b);
    }
    g_trace_pending.clear();
    return STB_OK;
}

stb_status check_workspace(void *ws, size_t bytes, size_t need) {
    if (!ws) return fail(STB_ERR_WORKSPACE, "workspace is NULL (%zu bytes needed)", need);
    if (reinterpret_cast<uintptr_t>(ws) % 256)
        return fail(STB_ERR_WORKSPACE, "workspace is not 256-byte aligned");
    if (bytes < need)
        return fail(STB_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", bytes, need);
    return STB_OK;
}

int32_t *status_word(void *ws) { return static_cast<int32_t *>(ws); }

// --------------------------------------------------------------- quadrature --
// Golub-Welsch: the Gauss nodes are the eigenvalues of the symmetric
// tridiagonal Jacobi matrix of the three-term recurrence and the weights are
// mu0 times the squared first components of its normalised eigenvectors.
// The eigenproblem is solved by implicit QL iterations with Wilkinson shifts,
// carrying only the first row of the eigenvector matrix.
static void golub_welsch(int n, std::vector<double> diag, std::vector<double> off, double mu0,
                         double *x, double *w) {
    // off[i] couples i and i+1 (i = 0..n-2); off[n-1] = 0 is scratch.
    off.resize(n, 0.0);
    std::vector<double> z(n, 0.0);
    z[0] = 1.0;
    for (int l = 0; l < n; ++l) {
        for (int iter = 0; iter < 100; ++iter) {
            int m = l;
            for (; m < n - 1; ++m) {
                double dd = std::fabs(diag[m]) + std::fabs(diag[m + 1]);
                if (std::fabs(off[m]) <= 1e-17 * dd) break;
            }
            if (m == l) break;
            double g = (diag[l + 1] - diag[l]) / (2.0 * off[l]);
            double r = std::hypot(g, 1.0);
            g = diag[m] - diag[l] + off[l] / (g + std::copysign(r, g));
            double s = 1.0, c = 1.0, p = 0.0;
            int i = m - 1;
            bool deflated = false;
            for (; i >= l; --i) {
                double f = s * off[i], b = c * off[i];
                r = std::hypot(f, g);
                off[i + 1] = r;
                if (r == 0.0) {
                    diag[i + 1] -= p;
                    off[m] = 0.0;
                    deflated = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = diag[i + 1] - p;
                r = (diag[i] - g) * s + 2.0 * c * b;
                p = s * r;
                diag[i + 1] = g + p;
                g = c * r - b;
                double zf = z[i + 1];
                z[i + 1] = s * z[i] + c * zf;
                z[i] = c * z[i] - s * zf;
            }
            if (deflated) continue;
            diag[l] -= p;
            off[l] = g;
            off[m] = 0.0;
        }
    }
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return diag[a] < diag[b]; });
    for (int i = 0; i < n; ++i) {
        x[i] = diag[idx[i]];
        w[i] = mu0 * z[idx[i]] * z[idx[i]];
    }
}

void gauss_legendre01(int n, double *x, double *w) {
    // Legendre on [-1,1]: a_k = 0, b_k = k / sqrt(4k^2 - 1), mu0 = 2
    std::vector<double> a(n, 0.0), b(n > 1 ? n - 1 : 0);
    for (int k = 1; k < n; ++k) b[k - 1] = k / std::sqrt(4.0 * k * k - 1.0);
    golub_welsch(n, a, b, 2.0, x, w);
    for (int i = 0; i < n; ++i) {
        x[i] = 0.5 * (x[i] + 1.0);
        w[i] *= 0.5;
    }
}

void gauss_jacobi_x01(int n, double *x, double *w) {
    // Jacobi (alpha, beta) = (0, 1) on [-1,1], weight (1 + y):
    // a_k = 1 / ((2k+1)(2k+3)), b_k = sqrt(k (k+1)) / (2k+1), mu0 = 2;
    // y = 2x - 1 turns the weight into 4x dx on [0,1].
    std::vector<double> a(n), b(n > 1 ? n - 1 : 0);
    for (int k = 0; k < n; ++k) a[k] = 1.0 / ((2.0 * k + 1.0) * (2.0 * k + 3.0));
    for (int k = 1; k < n; ++k) b[k - 1] = std::sqrt(double(k) * (k + 1)) / (2.0 * k + 1.0);
    golub_welsch(n, a, b, 2.0, x, w);
    for (int i = 0; i < n; ++i) {
        x[i] = 0.5 * (x[i] + 1.0);
        w[i] *= 0.25;
    }
}

void triangle_rule(int q, std::vector<double> &s1, std::vector<double> &s2,
                   std::vector<double> &w) {
    std::vector<double> xj(q), wj(q), xl(q), wl(q);
    gauss_jacobi_x01(q, xj.data(), wj.data());
    gauss_legendre01(q, xl.data(), wl.data());
    s1.clear();
    s2.clear();
    w.clear();
    for (int a = 0; a < q; ++a)
        for (int b = 0; b < q; ++b) {
            s1.push_back(xj[a]);          // sigma1
            s2.push_back(xj[a] * xl[b]);  // sigma1 * sigma2
            w.push_back(wj[a] * wl[b]);
        }
}

int ss_rule_size(int cls, int m) {
    int m4 = m * m * m * m;
    return cls == PAIR_IDENTICAL ? 6 * m4 : cls == PAIR_EDGE ? 4 * m4 : cls == PAIR_VERTEX ? 2 * m4 : 0;
}

// One point of a regularised rule: (u0..u3) in [0,1]^4 of sub-domain `sub`
// -> (s, t) in T x T and the Jacobian of the map.
//  identical (6 cones of z = t - s by the signs of z1, z2, z1 - z2):
//      z = zeta * e_sub(u0), s = corner_sub(z) + (1 - zeta)(p1, p1 p2),
//      jac = zeta (1 - zeta)^2 p1              [u = (zeta, u0', p1, p2)]
//  edge (4 cones of (t1 - s1, s2, t2), shared edge s2 = t2 = 0):
//      jac = zeta^2 (1 - zeta) [* a]
//  vertex (2 orderings of the Duffy radii, shared vertex s = t = 0):
//      jac = zeta^3 a
static void ss_point(int cls, int sub, const double u[4], double st[4], double &jac,
                     double *diff = nullptr) {
    const double zt = u[0], L = 1.0 - zt;
    if (cls == PAIR_IDENTICAL) {
        const double v = u[1], p1 = u[2], p2 = u[3];
        double z1, z2, c1, c2;
        switch (sub) {
            case 0: z1 = zt;            z2 = zt * v;         c1 = 0.0;     c2 = 0.0;  break;
            case 1: z1 = zt * v;        z2 = zt;             c1 = z2 - z1; c2 = 0.0;  break;
            case 2: z1 = zt * v;        z2 = zt * (v - 1.0); c1 = -z2;     c2 = -z2;  break;
            case 3: z1 = -zt * v;       z2 = zt * (1.0 - v); c1 = z2 - z1; c2 = 0.0;  break;
            case 4: z1 = -zt * v;       z2 = -zt;            c1 = -z2;     c2 = -z2;  break;
            default: z1 = -zt;          z2 = -zt * v;        c1 = -z1;     c2 = -z2;  break;
        }
        st[0] = c1 + L * p1;
        st[1] = c2 + L * p1 * p2;
        st[2] = st[0] + z1;
        st[3] = st[1] + z2;
        jac = zt * L * L * p1;
        if (diff) {
            diff[0] = z1;
            diff[1] = z2;
            diff[2] = diff[3] = 0.0;
        }
    } else if (cls == PAIR_EDGE) {
        const double a = u[1], b = u[2], sg = u[3];
        double s1, s2, t2, du;  // du = t1 - s1
        switch (sub) {
            case 0:  du = zt * a;        s2 = zt * (1.0 - a);     t2 = zt * b;          s1 = s2 + L * sg;      jac = zt * zt * L;     break;
            case 1:  du = zt * a * b;    s2 = zt * a * (1.0 - b); t2 = zt;              s1 = zt - du + L * sg; jac = zt * zt * L * a; break;
            case 2:  du = -zt * a * b;   s2 = zt;                 t2 = zt * a * (1.0 - b); s1 = zt + L * sg;   jac = zt * zt * L * a; break;
            default: du = -zt * a;       s2 = zt * b;             t2 = zt * (1.0 - a);  s1 = zt + L * sg;      jac = zt * zt * L;     break;
        }
        st[0] = s1;
        st[1] = s2;
        st[2] = s1 + du;
        st[3] = t2;
        if (diff) {
            diff[0] = du;
            diff[1] = s2;
            diff[2] = t2;
            diff[3] = 0.0;
        }
    } else {  // vertex
        const double a = u[1], p2 = u[2], q2 = u[3];
        const double S = sub == 0 ? zt : zt * a, R = sub == 0 ? zt * a : zt;
        st[0] = S;
        st[1] = S * p2;
        st[2] = R;
        st[3] = R * q2;
        jac = zt * zt * zt * a;
        if (diff)
            for (int i = 0; i < 4; ++i) diff[i] = st[i];
    }
}

void ss_rule_diff(int cls, int m, std::vector<double> &p0, std::vector<double> &p1,
                  std::vector<double> &p2, std::vector<double> &p3, std::vector<double> &w) {
    std::vector<double> g(m), gw(m);
    gauss_legendre01(m, g.data(), gw.data());
    int nsub = cls == PAIR_IDENTICAL ? 6 : cls == PAIR_EDGE ? 4 : 2;
    p0.clear(); p1.clear(); p2.clear(); p3.clear(); w.clear();
    for (int sub = 0; sub < nsub; ++sub)
        for (int i0 = 0; i0 < m; ++i0)
            for (int i1 = 0; i1 < m; ++i1)
                for (int i2 = 0; i2 < m; ++i2)
                    for (int i3 = 0; i3 < m; ++i3) {
                        double u[4] = {g[i0], g[i1], g[i2], g[i3]}, st[4], jac, df[4];
                        ss_point(cls, sub, u, st, jac, df);
                        p0.push_back(df[0]);
                        p1.push_back(df[1]);
                        p2.push_back(df[2]);
                        p3.push_back(df[3]);
                        w.push_back(gw[i0] * gw[i1] * gw[i2] * gw[i3] * jac);
                    }
}

void ss_rule(int cls, int m, std::vector<double> &s1, std::vector<double> &s2,
             std::vector<double> &t1, std::vector<double> &t2, std::vector<double> &w) {
    std::vector<double> g(m), gw(m);
    gauss_legendre01(m, g.data(), gw.data());
    int nsub = cls == PAIR_IDENTICAL ? 6 : cls == PAIR_EDGE ? 4 : 2;
    s1.clear(); s2.clear(); t1.clear(); t2.clear(); w.clear();
    for (int sub = 0; sub < nsub; ++sub)
        for (int i0 = 0; i0 < m; ++i0)
            for (int i1 = 0; i1 < m; ++i1)
                for (int i2 = 0; i2 < m; ++i2)
                    for (int i3 = 0; i3 < m; ++i3) {
                        double u[4] = {g[i0], g[i1], g[i2], g[i3]}, st[4], jac;
                        ss_point(cls, sub, u, st, jac);
                        s1.push_back(st[0]);
                        s2.push_back(st[1]);
                        t1.push_back(st[2]);
                        t2.push_back(st[3]);
                        w.push_back(gw[i0] * gw[i1] * gw[i2] * gw[i3] * jac);
                    }
}

}  // namespace stb

using namespace stb;

// ------------------------------------------------------------------ C ABI ----
extern "C" {

stb_params stb_default_params(double alpha, double T, int32_t n_steps) {
    stb_params p;
    p.alpha = alpha;
    p.T = T;
    p.n_steps = n_steps;
    p.quad_regular = 3;
    p.quad_singular = 4;
    p.precision = STB_PREC_FP64;
    p.storage = STB_STORE_F64;
    p.flags = 0;
    return p;
}

const char *stb_status_string(stb_status s) {
    switch (s) {
        case STB_OK: return "ok";
        case STB_ERR_INVALID_ARG: return "invalid argument";
        case STB_ERR_BAD_MESH: return "bad mesh";
        case STB_ERR_NOMEM: return "out of memory";
        case STB_ERR_CUDA: return "CUDA error";
        case STB_ERR_NOT_SPD: return "V^0 not positive definite";
        case STB_ERR_NOT_CONVERGED: return "not converged";
        case STB_ERR_TIMEOUT: return "bounded device wait expired";
        case STB_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
        default: return "unknown status";
    }
}

const char *stb_last_error_message(void) { return t_last_error.c_str(); }

int64_t stb_launch_count(void) { return g_launches.load(); }

stb_status stb_mesh_create(const double *nodes, int64_t n_nodes, const int32_t *tris,
                           int64_t n_tris, stb_mesh **out) {
    if (!out) return fail(STB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!nodes || !tris || n_nodes < 3 || n_tris < 4 || n_tris > (int64_t)1 << 24)
        return fail(STB_ERR_INVALID_ARG, "need nodes, tris, n_nodes >= 3, 4 <= n_tris <= 2^24");
    for (int64_t i = 0; i < 3 * n_nodes; ++i)
        if (!std::isfinite(nodes[i])) return fail(STB_ERR_BAD_MESH, "node coordinate %lld is not finite", (long long)i);
    // triangles: valid, distinct indices, positive area
    double ext = 0.0;
    for (int64_t i = 0; i < 3 * n_nodes; ++i) ext = std::max(ext, std::fabs(nodes[i]));
    for (int64_t e = 0; e < n_tris; ++e) {
        const int32_t *t = tris + 3 * e;
        for (int k = 0; k < 3; ++k)
            if (t[k] < 0 || t[k] >= n_nodes)
                return fail(STB_ERR_BAD_MESH, "triangle %lld has vertex index %d out of range", (long long)e, t[k]);
        if (t[0] == t[1] || t[1] == t[2] || t[0] == t[2])
            return fail(STB_ERR_BAD_MESH, "triangle %lld repeats a vertex", (long long)e);
        const double *a = nodes + 3 * t[0], *b = nodes + 3 * t[1], *c = nodes + 3 * t[2];
        double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double n[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
        double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(len > 1e-24 * (ext * ext + 1e-300)))
            return fail(STB_ERR_BAD_MESH, "triangle %lld is degenerate", (long long)e);
    }
    // closed, consistently oriented, edge-manifold: every directed edge once,
    // together with its reverse
    std::unordered_map<uint64_t, int32_t> dir;
    dir.reserve(3 * n_tris * 2);
    for (int64_t e = 0; e < n_tris; ++e)
        for (int k = 0; k < 3; ++k) {
            uint64_t u = tris[3 * e + k], v = tris[3 * e + (k + 1) % 3];
            if (!dir.emplace(u * (uint64_t)n_nodes + v, (int32_t)e).second)
                return fail(STB_ERR_BAD_MESH, "edge (%llu,%llu) is used twice in the same direction",
                            (unsigned long long)u, (unsigned long long)v);
        }
    for (auto &kv : dir) {
        uint64_t u = kv.first / n_nodes, v = kv.first % n_nodes;
        if (!dir.count(v * (uint64_t)n_nodes + u))
            return fail(STB_ERR_BAD_MESH, "edge (%llu,%llu) has no opposite neighbour: surface not closed or not oriented",
                        (unsigned long long)u, (unsigned long long)v);
    }
    // unordered touching pairs (a <= b), via the node -> triangle incidence
    std::vector<std::vector<int32_t>> inc(n_nodes);
    for (int64_t e = 0; e < n_tris; ++e)
        for (int k = 0; k < 3; ++k) inc[tris[3 * e + k]].push_back((int32_t)e);
    int64_t n_touch = 0;
    std::vector<int32_t> seen;
    for (int64_t a = 0; a < n_tris; ++a) {
        seen.clear();
        for (int k = 0; k < 3; ++k)
            for (int32_t b : inc[tris[3 * a + k]])
                if (b >= a) seen.push_back(b);
        std::sort(seen.begin(), seen.end());
        n_touch += std::unique(seen.begin(), seen.end()) - seen.begin();
    }
    stb_mesh *M = new (std::nothrow) stb_mesh;
    if (!M) return fail(STB_ERR_NOMEM, "mesh object");
    M->m.n_nodes = n_nodes;
    M->m.n_tris = n_tris;
    M->m.n_touch = n_touch;
    M->m.nodes.assign(nodes, nodes + 3 * n_nodes);
    M->m.tris.assign(tris, tris + 3 * n_tris);
    cudaError_t e1 = cudaMalloc(&M->m.d_nodes, sizeof(double) * 3 * n_nodes);
    cudaError_t e2 = e1 == cudaSuccess ? cudaMalloc(&M->m.d_tris, sizeof(int32_t) * 3 * n_tris) : e1;
    if (e2 != cudaSuccess) {
        stb_mesh_destroy(M);
        return e2 == cudaErrorMemoryAllocation ? fail(STB_ERR_NOMEM, "device mesh arrays")
                                               : cuda_fail(e2, "cudaMalloc(mesh)");
    }
    cudaError_t e3 = cudaMemcpy(M->m.d_nodes, nodes, sizeof(double) * 3 * n_nodes, cudaMemcpyHostToDevice);
    if (e3 == cudaSuccess)
        e3 = cudaMemcpy(M->m.d_tris, tris, sizeof(int32_t) * 3 * n_tris, cudaMemcpyHostToDevice);
    if (e3 != cudaSuccess) {
        stb_mesh_destroy(M);
        return cuda_fail(e3, "cudaMemcpy(mesh)");
    }
    *out = M;
    return STB_OK;
}

void stb_mesh_destroy(stb_mesh *M) {
    if (!M) return;
    if (M->m.d_nodes) cudaFree(M->m.d_nodes);
    if (M->m.d_tris) cudaFree(M->m.d_tris);
    delete M;
}

stb_status stb_mesh_info(const stb_mesh *M, int64_t *n_nodes, int64_t *n_tris, int64_t *n_touch) {
    if (!M) return fail(STB_ERR_INVALID_ARG, "mesh is NULL");
    if (n_nodes) *n_nodes = M->m.n_nodes;
    if (n_tris) *n_tris = M->m.n_tris;
    if (n_touch) *n_touch = M->m.n_touch;
    return STB_OK;
}

stb_status stb_trace_enable(int32_t on) {
    g_trace_on.store(on != 0);
    return STB_OK;
}

stb_status stb_trace_reset(void) {
    stb_status st = trace_drain();
    std::lock_guard<std::mutex> lk(g_trace_mu);
    g_trace_acc.clear();
    return st;
}

stb_status stb_trace_read(stb_trace_entry *out, int32_t max_entries, int32_t *n_entries) {
    if (!n_entries || (max_entries > 0 && !out)) return fail(STB_ERR_INVALID_ARG, "invalid argument");
    stb_status st = trace_drain();
    if (st) return st;
    std::lock_guard<std::mutex> lk(g_trace_mu);
    int32_t n = 0;
    for (auto &kv : g_trace_acc) {
        if (n < max_entries) {
            std::memset(out[n].name, 0, sizeof out[n].name);
            std::strncpy(out[n].name, kv.first.c_str(), sizeof out[n].name - 1);
            out[n].launches = kv.second.first;
            out[n].total_ms = kv.second.second;
        }
        ++n;
    }
    *n_entries = n;
    return STB_OK;
}

stb_status stb_workspace_status(const void *ws, stb_stream stream) {
    if (!ws) return fail(STB_ERR_INVALID_ARG, "workspace is NULL");
    int32_t st = 0;
    STB_CUDA(cudaMemcpyAsync(&st, ws, sizeof st, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    STB_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (st != STB_OK) return fail(st, "device status: %s", stb_status_string(st));
    return STB_OK;
}

}  // extern "C"
