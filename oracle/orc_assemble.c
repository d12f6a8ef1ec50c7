/*
 * orc_assemble.c -- mesh geometry, pair classification and the assembly of
 * the block lower-triangular Toeplitz matrices V_h and K_h with piecewise
 * constant test and trial functions (TEST INFRASTRUCTURE ONLY; see orc.h).
 *
 * Follows Sec. 3.1-3.2 (blocks V^d, K^d; eq. vd, eq. V0, eq. K_d, eq. K0),
 * Sec. 5 (loop over time levels i_t outermost, then test and trial elements;
 * the scatter of one time level into up to three blocks, Table deltad), and
 * eq. quad_reg / eq. quad_duffy for the spatial integrals.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "orc.h"

/* Area Delta_j and outward unit normal n_j = (v1-v0) x (v2-v0) / |.| (Sec. 3,
 * eq. quad_reg uses Delta_j; n_y of Sec. 2). */
int orc_triangle_geometry(const double *nodes, int64_t n_nodes,
                          const int32_t *tris, int64_t E, double *area,
                          double *normal)
{
    for (int64_t e = 0; e < E; ++e) {
        int32_t i0 = tris[3 * e], i1 = tris[3 * e + 1], i2 = tris[3 * e + 2];
        if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= n_nodes || i1 >= n_nodes ||
            i2 >= n_nodes)
            return -1;
        const double *a = nodes + 3 * i0, *b = nodes + 3 * i1, *c = nodes + 3 * i2;
        double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double n[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2],
                       u[0] * v[1] - u[1] * v[0]};
        double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(len > 0.0))
            return -1;
        area[e] = 0.5 * len;
        if (normal) {
            normal[3 * e] = n[0] / len;
            normal[3 * e + 1] = n[1] / len;
            normal[3 * e + 2] = n[2] / len;
        }
    }
    return 0;
}

/* Class of the pair (l, j) from shared vertex indices, and the local vertex
 * orders ol, oj used with chi: shared vertices first and in the same order.
 *   identical: both keep the stored order;
 *   edge     : ol rotates l so its shared edge is (v0, v1) in l's cyclic
 *              order; oj lists the same two vertices, then j's third one;
 *   vertex   : both rotate (keeping their cyclic order) the shared vertex to
 *              position 0;
 *   disjoint : stored orders.                                               */
int orc_pair_class(const int32_t *tl, const int32_t *tj, int32_t *ol,
                   int32_t *oj)
{
    int shared_l[3] = {0, 0, 0}, nshared = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (tl[a] == tj[b]) {
                shared_l[a] = 1;
                ++nshared;
            }
    for (int a = 0; a < 3; ++a) {
        ol[a] = a;
        oj[a] = a;
    }
    if (nshared == 3)
        return ORC_IDENTICAL;
    if (nshared == 0)
        return ORC_DISJOINT;
    if (nshared == 2) {
        int k = 0;
        while (!(shared_l[k] && shared_l[(k + 1) % 3]))
            ++k;
        for (int a = 0; a < 3; ++a)
            ol[a] = (k + a) % 3;
        int used[3] = {0, 0, 0};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 3; ++b)
                if (tj[b] == tl[ol[a]]) {
                    oj[a] = b;
                    used[b] = 1;
                }
        for (int b = 0; b < 3; ++b)
            if (!used[b])
                oj[2] = b;
        return ORC_EDGE;
    }
    int kl = 0, kj = 0;
    while (!shared_l[kl])
        ++kl;
    while (tj[kj] != tl[kl])
        ++kj;
    for (int a = 0; a < 3; ++a) {
        ol[a] = (kl + a) % 3;
        oj[a] = (kj + a) % 3;
    }
    return ORC_VERTEX;
}

/* chi(s) = P0 + s1 (P1 - P0) + s2 (P2 - P1) */
static void chi(const double *P0, const double *P1, const double *P2,
                double s1, double s2, double *x)
{
    for (int c = 0; c < 3; ++c)
        x[c] = P0[c] + s1 * (P1[c] - P0[c]) + s2 * (P2[c] - P1[c]);
}

/* Quadrature points of one pair in physical space: rho_q, rn_q, weight w_q
 * (weights include 4 Delta_l Delta_j). */
typedef struct {
    int n;
    double *rho, *rn, *w;
    int cls;
    /* optional (lam[0] != NULL): barycentric coordinates of y in the trial
     * triangle and the nodes they belong to (piecewise linear trial space) */
    double *lam[3];
    int32_t node[3];
    /* optional (lamx[0] != NULL): the same for x in the test triangle */
    double *lamx[3];
    int32_t nodex[3];
} pair_points;

typedef struct {
    int q_reg, m_ss, nreg;
    double *rs1, *rs2, *rw;                   /* triangle rule           */
    int nss[4];
    double *ss[4][5];                         /* s1 s2 t1 t2 w per class */
} rules;

static int rules_init(rules *R, int q_reg, int m_ss)
{
    memset(R, 0, sizeof(*R));
    R->q_reg = q_reg;
    R->m_ss = m_ss;
    R->nreg = q_reg * q_reg;
    R->rs1 = malloc(sizeof(double) * R->nreg);
    R->rs2 = malloc(sizeof(double) * R->nreg);
    R->rw = malloc(sizeof(double) * R->nreg);
    if (orc_triangle_rule(q_reg, R->rs1, R->rs2, R->rw))
        return -1;
    for (int cls = 1; cls <= 3; ++cls) {
        int n = orc_ss_rule_size(cls, m_ss);
        R->nss[cls] = n;
        for (int c = 0; c < 5; ++c)
            R->ss[cls][c] = malloc(sizeof(double) * n);
        if (orc_ss_rule(cls, m_ss, R->ss[cls][0], R->ss[cls][1], R->ss[cls][2],
                        R->ss[cls][3], R->ss[cls][4]))
            return -1;
    }
    return 0;
}

static void rules_free(rules *R)
{
    free(R->rs1);
    free(R->rs2);
    free(R->rw);
    for (int cls = 1; cls <= 3; ++cls)
        for (int c = 0; c < 5; ++c)
            free(R->ss[cls][c]);
}

/* A touching pair's regularised rule is built once for the ordered pair
 * (a, b) = (min(l, j), max(l, j)) and used for both entries (l, j) and
 * (j, l) with the roles of x and y exchanged, so that V^d (whose kernel only
 * depends on |x - y|) is symmetric up to rounding, as the continuous
 * operator's Galerkin matrix is. */
static void pair_points_build(const rules *R, const double *nodes,
                              const int32_t *tris, const double *area,
                              const double *normal, int64_t l, int64_t j,
                              pair_points *pp)
{
    const double *n = normal + 3 * j;
    double scale = 4.0 * area[l] * area[j];
    int k = 0;
    int64_t ia = l < j ? l : j, ib = l < j ? j : l;
    int32_t oa[3], ob[3];
    const int32_t *ta = tris + 3 * ia, *tb = tris + 3 * ib;
    int cls = orc_pair_class(ta, tb, oa, ob);
    pp->cls = cls;
    if (cls == ORC_DISJOINT) {
        const int32_t *tl = tris + 3 * l, *tj = tris + 3 * j;
        for (int a = 0; a < R->nreg; ++a)
            for (int b = 0; b < R->nreg; ++b) {
                double x[3], y[3];
                chi(nodes + 3 * tl[0], nodes + 3 * tl[1], nodes + 3 * tl[2], R->rs1[a],
                    R->rs2[a], x);
                chi(nodes + 3 * tj[0], nodes + 3 * tj[1], nodes + 3 * tj[2], R->rs1[b],
                    R->rs2[b], y);
                double r0 = x[0] - y[0], r1 = x[1] - y[1], r2 = x[2] - y[2];
                pp->rho[k] = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
                pp->rn[k] = r0 * n[0] + r1 * n[1] + r2 * n[2];
                pp->w[k] = scale * R->rw[a] * R->rw[b];
                if (pp->lam[0]) { /* chi = (1-s1) P0 + (s1-s2) P1 + s2 P2 */
                    pp->lam[0][k] = 1.0 - R->rs1[b];
                    pp->lam[1][k] = R->rs1[b] - R->rs2[b];
                    pp->lam[2][k] = R->rs2[b];
                }
                if (pp->lamx[0]) {
                    pp->lamx[0][k] = 1.0 - R->rs1[a];
                    pp->lamx[1][k] = R->rs1[a] - R->rs2[a];
                    pp->lamx[2][k] = R->rs2[a];
                }
                ++k;
            }
        for (int c = 0; c < 3; ++c) {
            pp->node[c] = tj[c];
            pp->nodex[c] = tl[c];
        }
    } else {
        const double *Pa[3], *Pb[3];
        for (int c = 0; c < 3; ++c) {
            Pa[c] = nodes + 3 * ta[oa[c]];
            Pb[c] = nodes + 3 * tb[ob[c]];
        }
        double *const *t = R->ss[cls];
        for (int q = 0; q < R->nss[cls]; ++q) {
            double p[3], pb[3], x[3], y[3];
            chi(Pa[0], Pa[1], Pa[2], t[0][q], t[1][q], p);
            chi(Pb[0], Pb[1], Pb[2], t[2][q], t[3][q], pb);
            for (int c = 0; c < 3; ++c) {
                x[c] = l == ia ? p[c] : pb[c];
                y[c] = l == ia ? pb[c] : p[c];
            }
            double r0 = x[0] - y[0], r1 = x[1] - y[1], r2 = x[2] - y[2];
            pp->rho[k] = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
            pp->rn[k] = r0 * n[0] + r1 * n[1] + r2 * n[2];
            pp->w[k] = scale * t[4][q];
            if (pp->lam[0]) { /* y on b (coordinates t2, t3) when l = a, else on a */
                double u1 = l == ia ? t[2][q] : t[0][q], u2 = l == ia ? t[3][q] : t[1][q];
                pp->lam[0][k] = 1.0 - u1;
                pp->lam[1][k] = u1 - u2;
                pp->lam[2][k] = u2;
            }
            if (pp->lamx[0]) { /* x on a (coordinates t0, t1) when l = a, else on b */
                double u1 = l == ia ? t[0][q] : t[2][q], u2 = l == ia ? t[1][q] : t[3][q];
                pp->lamx[0][k] = 1.0 - u1;
                pp->lamx[1][k] = u1 - u2;
                pp->lamx[2][k] = u2;
            }
            ++k;
        }
        for (int c = 0; c < 3; ++c) {
            pp->node[c] = l == ia ? tb[ob[c]] : ta[oa[c]];
            pp->nodex[c] = l == ia ? ta[oa[c]] : tb[ob[c]];
        }
    }
    pp->n = k;
}

/* Spatial sums of one pair at one time level (level < 0: the delta = 0
 * singular integrand G^{dtau}(., 0), alpha dG^{dtau}/dn_y(., 0)).
 * For an identical pair of flat triangles r . n_y vanishes identically, so
 * its K sums are exactly zero. */
static void level_sums(const pair_points *pp, int level, double h,
                       double alpha, double *sv, double *sk)
{
    double v = 0.0, k = 0.0, delta = level < 0 ? 0.0 : level * h;
    for (int q = 0; q < pp->n; ++q) {
        if (level < 0) {
            v += pp->w[q] * orc_G_dtau(pp->rho[q], 0.0, alpha);
            k += pp->w[q] * orc_dn_G_dtau(pp->rn[q], pp->rho[q], 0.0, alpha);
        } else {
            v += pp->w[q] * orc_G_dtau_dt(pp->rho[q], delta, alpha);
            k += pp->w[q] * orc_dn_G_dtau_dt(pp->rn[q], pp->rho[q], delta, alpha);
        }
    }
    *sv = v;
    *sk = pp->cls == ORC_IDENTICAL ? 0.0 : k;
}

/* K sums of one pair at one level weighted by the trial triangle's
 * barycentric coordinates: sk[v] = sum_q w_q lam_v(y_q) alpha dG/dn_y(...). */
static void level_sums_k1(const pair_points *pp, int level, double h,
                          double alpha, double *sk)
{
    double delta = level < 0 ? 0.0 : level * h;
    sk[0] = sk[1] = sk[2] = 0.0;
    if (pp->cls == ORC_IDENTICAL)
        return;
    for (int q = 0; q < pp->n; ++q) {
        double k = level < 0 ? orc_dn_G_dtau(pp->rn[q], pp->rho[q], 0.0, alpha)
                             : orc_dn_G_dtau_dt(pp->rn[q], pp->rho[q], delta, alpha);
        for (int v = 0; v < 3; ++v)
            sk[v] += pp->w[q] * pp->lam[v][q] * k;
    }
}

static int geometry_alloc(const double *nodes, int64_t n_nodes,
                          const int32_t *tris, int64_t E, double **area,
                          double **normal)
{
    *area = malloc(sizeof(double) * E);
    *normal = malloc(sizeof(double) * 3 * E);
    return orc_triangle_geometry(nodes, n_nodes, tris, E, *area, *normal);
}

int orc_pair_sums(const double *nodes, int64_t n_nodes, const int32_t *tris,
                  int64_t E, int64_t l, int64_t j, double alpha, double h,
                  int n_levels, int q_reg, int m_ss, double *SV, double *SK)
{
    if (l < 0 || j < 0 || l >= E || j >= E || n_levels < 1)
        return -1;
    rules R;
    double *area = NULL, *normal = NULL;
    int rc = -1;
    if (rules_init(&R, q_reg, m_ss))
        goto done;
    if (geometry_alloc(nodes, n_nodes, tris, E, &area, &normal))
        goto done;
    int nmax = R.nreg * R.nreg;
    for (int c = 1; c <= 3; ++c)
        if (R.nss[c] > nmax)
            nmax = R.nss[c];
    pair_points pp;
    memset(&pp, 0, sizeof pp);
    pp.rho = malloc(sizeof(double) * nmax);
    pp.rn = malloc(sizeof(double) * nmax);
    pp.w = malloc(sizeof(double) * nmax);
    pair_points_build(&R, nodes, tris, area, normal, l, j, &pp);
    for (int i = 0; i < n_levels; ++i)
        level_sums(&pp, i, h, alpha, SV + i, SK + i);
    level_sums(&pp, -1, h, alpha, SV + n_levels, SK + n_levels);
    free(pp.rho);
    free(pp.rn);
    free(pp.w);
    rc = 0;
done:
    rules_free(&R);
    free(area);
    free(normal);
    return rc;
}

/* Add `value` of time level i_t to the blocks it feeds (Table deltad):
 * -value to d = i_t - 1, +2 value to d = i_t (i_t >= 1; +value at i_t = 0),
 * -value to d = i_t + 1. */
static void scatter(double *row_blocks, int64_t E, int n_steps, int i_t,
                    int64_t j, double value)
{
    if (i_t > 0) {
        row_blocks[(int64_t)(i_t - 1) * E + j] -= value;
        if (i_t < n_steps)
            row_blocks[(int64_t)i_t * E + j] += 2.0 * value;
    } else {
        row_blocks[j] += value;
    }
    if (i_t < n_steps - 1)
        row_blocks[(int64_t)(i_t + 1) * E + j] -= value;
}

int orc_assemble_rows(const double *nodes, int64_t n_nodes,
                      const int32_t *tris, int64_t E, double alpha, double T,
                      int32_t n_steps, int32_t q_reg, int32_t m_ss,
                      const int64_t *rows, int64_t n_rows, double *V,
                      double *K, double *SV, double *SK)
{
    if (E < 1 || n_steps < 1 || !(alpha > 0.0) || !(T > 0.0) || n_rows < 0)
        return -1;
    for (int64_t r = 0; r < n_rows; ++r)
        if (rows[r] < 0 || rows[r] >= E)
            return -1;
    rules R;
    double *area = NULL, *normal = NULL;
    int rc = -1;
    if (rules_init(&R, q_reg, m_ss))
        goto done;
    if (geometry_alloc(nodes, n_nodes, tris, E, &area, &normal))
        goto done;
    double h = T / n_steps;
    memset(V, 0, sizeof(double) * n_rows * n_steps * E);
    memset(K, 0, sizeof(double) * n_rows * n_steps * E);
    int nmax = R.nreg * R.nreg;
    for (int c = 1; c <= 3; ++c)
        if (R.nss[c] > nmax)
            nmax = R.nss[c];
    pair_points pp;
    memset(&pp, 0, sizeof pp);
    pp.rho = malloc(sizeof(double) * nmax);
    pp.rn = malloc(sizeof(double) * nmax);
    pp.w = malloc(sizeof(double) * nmax);
    int64_t sstride = (int64_t)(n_steps + 2) * E;
    for (int i_t = 0; i_t <= n_steps; ++i_t) {
        for (int64_t r = 0; r < n_rows; ++r) {
            int64_t l = rows[r];
            double *Vr = V + r * (int64_t)n_steps * E;
            double *Kr = K + r * (int64_t)n_steps * E;
            for (int64_t j = 0; j < E; ++j) {
                pair_points_build(&R, nodes, tris, area, normal, l, j, &pp);
                double sv, sk;
                level_sums(&pp, i_t, h, alpha, &sv, &sk);
                scatter(Vr, E, n_steps, i_t, j, sv);
                scatter(Kr, E, n_steps, i_t, j, sk);
                if (SV) {
                    SV[r * sstride + (int64_t)i_t * E + j] = sv;
                    SK[r * sstride + (int64_t)i_t * E + j] = sk;
                }
                if (i_t == 0) {
                    /* eq. V0 / eq. K0: the h G^{dtau}(., 0) term of block 0 */
                    double sv0, sk0;
                    level_sums(&pp, -1, h, alpha, &sv0, &sk0);
                    Vr[j] += h * sv0;
                    Kr[j] += h * sk0;
                    if (SV) {
                        SV[r * sstride + (int64_t)(n_steps + 1) * E + j] = sv0;
                        SK[r * sstride + (int64_t)(n_steps + 1) * E + j] = sk0;
                    }
                }
            }
        }
    }
    free(pp.rho);
    free(pp.rn);
    free(pp.w);
    rc = 0;
done:
    rules_free(&R);
    free(area);
    free(normal);
    return rc;
}

/* Rows of all blocks of K_h with the piecewise-linear trial space of Sec. 3.2
 * (the paper's discretisation of the double layer): K1^d[l][i] =
 * int_{gamma_l} int_{Gamma_h} phi_i(y) K^d(x - y), i over the mesh nodes, as
 * second differences of the level sums (Table deltad, eq. K_d / eq. K0).
 * K1: [n_rows][n_steps][n_nodes]. */
int orc_assemble_k1_rows(const double *nodes, int64_t n_nodes,
                         const int32_t *tris, int64_t E, double alpha, double T,
                         int32_t n_steps, int32_t q_reg, int32_t m_ss,
                         const int64_t *rows, int64_t n_rows, double *K1)
{
    if (E < 1 || n_nodes < 3 || n_steps < 1 || !(alpha > 0.0) || !(T > 0.0) || n_rows < 0)
        return -1;
    for (int64_t r = 0; r < n_rows; ++r)
        if (rows[r] < 0 || rows[r] >= E)
            return -1;
    rules R;
    double *area = NULL, *normal = NULL;
    int rc = -1;
    if (rules_init(&R, q_reg, m_ss))
        goto done;
    if (geometry_alloc(nodes, n_nodes, tris, E, &area, &normal))
        goto done;
    double h = T / n_steps;
    memset(K1, 0, sizeof(double) * n_rows * n_steps * n_nodes);
    int nmax = R.nreg * R.nreg;
    for (int c = 1; c <= 3; ++c)
        if (R.nss[c] > nmax)
            nmax = R.nss[c];
    pair_points pp;
    memset(&pp, 0, sizeof pp);
    pp.rho = malloc(sizeof(double) * nmax);
    pp.rn = malloc(sizeof(double) * nmax);
    pp.w = malloc(sizeof(double) * nmax);
    for (int v = 0; v < 3; ++v)
        pp.lam[v] = malloc(sizeof(double) * nmax);
    for (int i_t = 0; i_t <= n_steps; ++i_t) {
        for (int64_t r = 0; r < n_rows; ++r) {
            int64_t l = rows[r];
            double *Kr = K1 + r * (int64_t)n_steps * n_nodes;
            for (int64_t j = 0; j < E; ++j) {
                pair_points_build(&R, nodes, tris, area, normal, l, j, &pp);
                double sk[3];
                level_sums_k1(&pp, i_t, h, alpha, sk);
                for (int v = 0; v < 3; ++v)
                    scatter(Kr, n_nodes, n_steps, i_t, pp.node[v], sk[v]);
                if (i_t == 0) { /* eq. K0: the h dG^{dtau}/dn(., 0) term of block 0 */
                    level_sums_k1(&pp, -1, h, alpha, sk);
                    for (int v = 0; v < 3; ++v)
                        Kr[pp.node[v]] += h * sk[v];
                }
            }
        }
    }
    free(pp.rho);
    free(pp.rn);
    free(pp.w);
    for (int v = 0; v < 3; ++v)
        free(pp.lam[v]);
    rc = 0;
done:
    rules_free(&R);
    free(area);
    free(normal);
    return rc;
}

/* ---- hypersingular operator (Sec. 3.3) -------------------------------------
 * D_h = D_h^1 + D_h^2 on X_h^{1,0} x X_h^{1,0}, blocks [n_steps][N][N].
 *
 * D^{2,d}[i][j] = int int n_x . n_y phi_i(x) phi_j(y) D^{2,d}(x - y) with
 *   D^{2,0}(r) = alpha [G^{dtau}(r, 0) - G^{dtau}(r, h)],
 *   D^{2,d}(r) = alpha [2 G^{dtau}(r, dh) - G^{dtau}(r, (d+1)h) - G^{dtau}(r, (d-1)h)]
 * (eq. D2d with G^{dt} = -G^{dtau}; the delta = 0 value is the limit of
 * eq. G_dtau_lim_d), integrated by the same rules as V.  The test
 * triangles test_tris[0..n_test) add their pairs with every trial triangle
 * into D2 (not zeroed here), so that rows of triangles can be split across
 * threads and summed.                                                      */
int orc_assemble_d2_tris(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t E,
                         double alpha, double T, int32_t n_steps, int32_t q_reg, int32_t m_ss,
                         const int64_t *test_tris, int64_t n_test, double *D2)
{
    if (E < 1 || n_nodes < 3 || n_steps < 1 || !(alpha > 0.0) || !(T > 0.0) || n_test < 0)
        return -1;
    for (int64_t r = 0; r < n_test; ++r)
        if (test_tris[r] < 0 || test_tris[r] >= E)
            return -1;
    rules R;
    double *area = NULL, *normal = NULL;
    int rc = -1;
    if (rules_init(&R, q_reg, m_ss))
        goto done;
    if (geometry_alloc(nodes, n_nodes, tris, E, &area, &normal))
        goto done;
    double h = T / n_steps;
    int nmax = R.nreg * R.nreg;
    for (int c = 1; c <= 3; ++c)
        if (R.nss[c] > nmax)
            nmax = R.nss[c];
    pair_points pp;
    memset(&pp, 0, sizeof pp);
    pp.rho = malloc(sizeof(double) * nmax);
    pp.rn = malloc(sizeof(double) * nmax);
    pp.w = malloc(sizeof(double) * nmax);
    for (int v = 0; v < 3; ++v) {
        pp.lam[v] = malloc(sizeof(double) * nmax);
        pp.lamx[v] = malloc(sizeof(double) * nmax);
    }
    const int64_t NN = n_nodes * n_nodes;
    for (int64_t r = 0; r < n_test; ++r) {
        int64_t l = test_tris[r];
        for (int64_t j = 0; j < E; ++j) {
            pair_points_build(&R, nodes, tris, area, normal, l, j, &pp);
            const double nn = normal[3 * l] * normal[3 * j] + normal[3 * l + 1] * normal[3 * j + 1] +
                              normal[3 * l + 2] * normal[3 * j + 2];
            for (int i_t = 0; i_t <= n_steps; ++i_t) {
                /* S[a][b] = sum_q w_q lam_a(x_q) lam_b(y_q) G^{dtau}(rho_q, i_t h) */
                double S[3][3] = {{0}};
                for (int q = 0; q < pp.n; ++q) {
                    double g = pp.w[q] * orc_G_dtau(pp.rho[q], i_t * h, alpha);
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            S[a][b] += pp.lamx[a][q] * pp.lam[b][q] * g;
                }
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        double v = alpha * nn * S[a][b];
                        int64_t ij = (int64_t)pp.nodex[a] * n_nodes + pp.node[b];
                        /* level i_t feeds d = i_t (+2, or +1 for i_t = 0), d = i_t - 1
                         * and d = i_t + 1 (-1 each) */
                        if (i_t == 0) {
                            D2[ij] += v;
                        } else if (i_t < n_steps) {
                            D2[(int64_t)i_t * NN + ij] += 2.0 * v;
                        }
                        if (i_t >= 1)
                            D2[(int64_t)(i_t - 1) * NN + ij] -= v;
                        if (i_t + 1 < n_steps)
                            D2[(int64_t)(i_t + 1) * NN + ij] -= v;
                    }
            }
        }
    }
    free(pp.rho);
    free(pp.rn);
    free(pp.w);
    for (int v = 0; v < 3; ++v) {
        free(pp.lam[v]);
        free(pp.lamx[v]);
    }
    rc = 0;
done:
    rules_free(&R);
    free(area);
    free(normal);
    return rc;
}

/* Surface curls of the hat functions, constant on each triangle:
 * curl phi_v = n x grad phi_v with grad phi_v = n x (P_{v+2} - P_{v+1}) / (2 Delta)
 * (the in-plane normal of the opposite edge, pointing to P_v, of length
 * 1 / height); curl[(3 m + v) * 3 + o] for vertex v of triangle m. */
int orc_surface_curls(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t E,
                      double *curl)
{
    double *area = NULL, *normal = NULL;
    if (geometry_alloc(nodes, n_nodes, tris, E, &area, &normal)) {
        free(area);
        free(normal);
        return -1;
    }
    for (int64_t m = 0; m < E; ++m) {
        const double *n = normal + 3 * m;
        for (int v = 0; v < 3; ++v) {
            const double *A = nodes + 3 * tris[3 * m + (v + 1) % 3];
            const double *B = nodes + 3 * tris[3 * m + (v + 2) % 3];
            double e[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]}, g[3];
            g[0] = (n[1] * e[2] - n[2] * e[1]) / (2.0 * area[m]);
            g[1] = (n[2] * e[0] - n[0] * e[2]) / (2.0 * area[m]);
            g[2] = (n[0] * e[1] - n[1] * e[0]) / (2.0 * area[m]);
            double *c = curl + (3 * m + v) * 3;
            c[0] = n[1] * g[2] - n[2] * g[1];
            c[1] = n[2] * g[0] - n[0] * g[2];
            c[2] = n[0] * g[1] - n[1] * g[0];
        }
    }
    free(area);
    free(normal);
    return 0;
}

/* D^{1,d} = T^T (alpha^2 V^d (x) I_3) T (eq. D_1_sp_trafo), T_o[m][j] the
 * o-th component of the surface curl of phi_j on triangle m; V [n_steps][E][E]
 * the single-layer blocks.  D1 [n_steps][N][N] is overwritten.             */
int orc_assemble_d1(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t E,
                    double alpha, int32_t n_steps, const double *V, double *D1)
{
    if (E < 1 || n_nodes < 3 || n_steps < 1)
        return -1;
    double *curl = malloc(sizeof(double) * 9 * E);
    double *Tm = calloc((size_t)3 * E * n_nodes, sizeof(double)); /* T [3][E][N] */
    double *W = malloc(sizeof(double) * 3 * E * n_nodes);          /* V T_o      */
    int rc = -1;
    if (!curl || !Tm || !W || orc_surface_curls(nodes, n_nodes, tris, E, curl))
        goto done;
    for (int64_t m = 0; m < E; ++m)
        for (int v = 0; v < 3; ++v)
            for (int o = 0; o < 3; ++o)
                Tm[((int64_t)o * E + m) * n_nodes + tris[3 * m + v]] += curl[(3 * m + v) * 3 + o];
    const int64_t NN = n_nodes * n_nodes, EE = E * E;
    for (int d = 0; d < n_steps; ++d) {
        const double *Vd = V + d * EE;
        for (int o = 0; o < 3; ++o)
            for (int64_t nn = 0; nn < E; ++nn)
                for (int64_t j = 0; j < n_nodes; ++j) {
                    double acc = 0.0;
                    for (int64_t m = 0; m < E; ++m)
                        acc += Vd[nn * E + m] * Tm[((int64_t)o * E + m) * n_nodes + j];
                    W[((int64_t)o * E + nn) * n_nodes + j] = acc;
                }
        double *Dd = D1 + d * NN;
        for (int64_t i = 0; i < n_nodes; ++i)
            for (int64_t j = 0; j < n_nodes; ++j) {
                double acc = 0.0;
                for (int o = 0; o < 3; ++o)
                    for (int64_t nn = 0; nn < E; ++nn)
                        acc += Tm[((int64_t)o * E + nn) * n_nodes + i] *
                               W[((int64_t)o * E + nn) * n_nodes + j];
                Dd[i * n_nodes + j] = alpha * alpha * acc;
            }
    }
    rc = 0;
done:
    free(curl);
    free(Tm);
    free(W);
    return rc;
}

/* ---- non-uniform time grids (Sec. 7: the antiderivatives carry over) -------
 * Time grid t_0 = 0 < t_1 < ... < t_n; blocks A^{k,i} (k >= i) of the block
 * lower-triangular matrices, packed at b(k,i) = k(k+1)/2 + i.  With
 * Phi = G^{dtau dt} (and its scaled normal derivative for K), whose second
 * derivative in delta is -G, the double time integral over
 * [t_k, t_{k+1}] x [t_i, t_{i+1}] is
 *   A^{k,i} = S(t_{k+1} - t_{i+1}) - S(t_k - t_{i+1}) - S(t_{k+1} - t_i) + S(t_k - t_i)
 * for k > i (S the pair's spatial sum of Phi; S(0) the delta -> 0 limit), and
 *   A^{k,k} = h_k S_*(0) - S(h_k) + S(0),   h_k = t_{k+1} - t_k
 * on the diagonal (eq. V0 / eq. K0 with the step h_k).                       */
static void level_sums_delta(const pair_points *pp, double delta, double alpha, double *sv,
                             double *sk)
{
    double v = 0.0, k = 0.0;
    for (int q = 0; q < pp->n; ++q) {
        v += pp->w[q] * orc_G_dtau_dt(pp->rho[q], delta, alpha);
        k += pp->w[q] * orc_dn_G_dtau_dt(pp->rn[q], pp->rho[q], delta, alpha);
    }
    *sv = v;
    *sk = pp->cls == ORC_IDENTICAL ? 0.0 : k;
}

int orc_assemble_rows_nu(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t E,
                         double alpha, const double *times, int32_t n_steps, int32_t q_reg,
                         int32_t m_ss, const int64_t *rows, int64_t n_rows, double *V, double *K)
{
    if (E < 1 || n_steps < 1 || !(alpha > 0.0) || n_rows < 0 || !times || times[0] != 0.0)
        return -1;
    for (int k = 0; k < n_steps; ++k)
        if (!(times[k + 1] > times[k]))
            return -1;
    for (int64_t r = 0; r < n_rows; ++r)
        if (rows[r] < 0 || rows[r] >= E)
            return -1;
    rules R;
    double *area = NULL, *normal = NULL;
    int rc = -1;
    if (rules_init(&R, q_reg, m_ss))
        goto done;
    if (geometry_alloc(nodes, n_nodes, tris, E, &area, &normal))
        goto done;
    const int64_t nblk = (int64_t)n_steps * (n_steps + 1) / 2;
    int nmax = R.nreg * R.nreg;
    for (int c = 1; c <= 3; ++c)
        if (R.nss[c] > nmax)
            nmax = R.nss[c];
    pair_points pp;
    memset(&pp, 0, sizeof pp);
    pp.rho = malloc(sizeof(double) * nmax);
    pp.rn = malloc(sizeof(double) * nmax);
    pp.w = malloc(sizeof(double) * nmax);
    for (int64_t r = 0; r < n_rows; ++r) {
        int64_t l = rows[r];
        double *Vr = V + r * nblk * E, *Kr = K + r * nblk * E;
        for (int64_t j = 0; j < E; ++j) {
            pair_points_build(&R, nodes, tris, area, normal, l, j, &pp);
            double s0v, s0k, ssv, ssk;
            level_sums_delta(&pp, 0.0, alpha, &s0v, &s0k);
            /* the delta = 0 singular integrand G^{dtau}(., 0) */
            ssv = 0.0;
            ssk = 0.0;
            for (int q = 0; q < pp.n; ++q) {
                ssv += pp.w[q] * orc_G_dtau(pp.rho[q], 0.0, alpha);
                ssk += pp.w[q] * orc_dn_G_dtau(pp.rn[q], pp.rho[q], 0.0, alpha);
            }
            if (pp.cls == ORC_IDENTICAL)
                ssk = 0.0;
            for (int k = 0; k < n_steps; ++k)
                for (int i = 0; i <= k; ++i) {
                    double v, kk;
                    if (i == k) {
                        double h = times[k + 1] - times[k], sv, sk;
                        level_sums_delta(&pp, h, alpha, &sv, &sk);
                        v = h * ssv - sv + s0v;
                        kk = h * ssk - sk + s0k;
                    } else {
                        double a1, b1, a2, b2, a3, b3, a4, b4;
                        level_sums_delta(&pp, times[k + 1] - times[i + 1], alpha, &a1, &b1);
                        level_sums_delta(&pp, times[k] - times[i + 1], alpha, &a2, &b2);
                        level_sums_delta(&pp, times[k + 1] - times[i], alpha, &a3, &b3);
                        level_sums_delta(&pp, times[k] - times[i], alpha, &a4, &b4);
                        v = a1 - a2 - a3 + a4;
                        kk = b1 - b2 - b3 + b4;
                    }
                    int64_t b = (int64_t)k * (k + 1) / 2 + i;
                    Vr[b * E + j] = v;
                    Kr[b * E + j] = kk;
                }
        }
    }
    free(pp.rho);
    free(pp.rn);
    free(pp.w);
    rc = 0;
done:
    rules_free(&R);
    free(area);
    free(normal);
    return rc;
}

