/*
 * orc_solve.c -- Dirichlet data projection, right-hand side (1/2 M_h + K_h) g,
 * block-Toeplitz matrix-vector product and block forward substitution for
 * V_h w = (1/2 M_h + K_h) g, plus the L2(Sigma_h) error of w_h
 * (TEST INFRASTRUCTURE ONLY; see orc.h).
 *
 * Sec. 3.4 (systems of linear equations), Sec. 6.1 (exterior heat source
 * data and the relative L2(Sigma_h) error).  With piecewise constant trial
 * functions for g the mass matrix is M_h = h blockdiag(diag(Delta_l)).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "orc.h"

static void chi_plain(const double *P0, const double *P1, const double *P2,
                      double s1, double s2, double *x)
{
    for (int c = 0; c < 3; ++c)
        x[c] = P0[c] + s1 * (P1[c] - P0[c]) + s2 * (P2[c] - P1[c]);
}

/* g_r(x, t) = sum_s weight_s G_alpha(x - y_s, t - t0_s) */
static double dirichlet_datum(const double *src, int32_t n_src, double alpha,
                              const double *x, double t)
{
    double g = 0.0;
    for (int s = 0; s < n_src; ++s) {
        const double *S = src + 5 * s;
        double d0 = x[0] - S[0], d1 = x[1] - S[1], d2 = x[2] - S[2];
        g += S[4] * orc_heat_kernel(sqrt(d0 * d0 + d1 * d1 + d2 * d2), t - S[3], alpha);
    }
    return g;
}

/* w_r(x, t) = alpha du/dn_x = sum_s weight_s alpha grad_x G . n_x
 *          = -sum_s weight_s G_alpha(x - y_s, t - t0_s) ((x - y_s) . n_x) / (2 (t - t0_s)) */
static double neumann_datum(const double *src, int32_t n_src, double alpha,
                            const double *x, const double *n, double t)
{
    double w = 0.0;
    for (int s = 0; s < n_src; ++s) {
        const double *S = src + 5 * s;
        double tau = t - S[3];
        if (tau <= 0.0)
            continue;
        double d0 = x[0] - S[0], d1 = x[1] - S[1], d2 = x[2] - S[2];
        double rho = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        double dn = d0 * n[0] + d1 * n[1] + d2 * n[2];
        w -= S[4] * orc_heat_kernel(rho, tau, alpha) * dn / (2.0 * tau);
    }
    return w;
}

/* L2 projection into piecewise constants: the element mean
 * g_{r,k,j} = (h Delta_j)^{-1} int_{t_k}^{t_{k+1}} int_{gamma_j} g_r,
 * by the conical rule of order q_space in space and n_time Gauss-Legendre
 * points per step (the paper only asks for rules of sufficiently high order). */
int orc_project_dirichlet(const double *nodes, int64_t n_nodes,
                          const int32_t *tris, int64_t E, double alpha,
                          double T, int32_t n_steps, const double *sources,
                          int32_t n_src, int32_t nrhs, int32_t q_space,
                          int32_t n_time, double *g)
{
    if (E < 1 || n_steps < 1 || nrhs < 1 || n_src < 1 || q_space < 1 ||
        q_space > 32 || n_time < 1 || n_time > 64)
        return -1;
    int nq = q_space * q_space;
    double *s1 = malloc(sizeof(double) * nq), *s2 = malloc(sizeof(double) * nq);
    double *sw = malloc(sizeof(double) * nq), tx[64], tw[64];
    int rc = -1;
    if (orc_triangle_rule(q_space, s1, s2, sw) || orc_gauss_legendre01(n_time, tx, tw))
        goto done;
    double h = T / n_steps;
    for (int r = 0; r < nrhs; ++r)
        for (int k = 0; k < n_steps; ++k)
            for (int64_t j = 0; j < E; ++j) {
                const int32_t *t3 = tris + 3 * j;
                double acc = 0.0;
                for (int a = 0; a < nq; ++a) {
                    double x[3];
                    chi_plain(nodes + 3 * t3[0], nodes + 3 * t3[1], nodes + 3 * t3[2],
                              s1[a], s2[a], x);
                    for (int b = 0; b < n_time; ++b)
                        acc += sw[a] * tw[b] *
                               dirichlet_datum(sources + (int64_t)r * n_src * 5, n_src,
                                               alpha, x, (k + tx[b]) * h);
                }
                /* (h Delta)^{-1} * (2 Delta) * h * acc */
                g[((int64_t)r * n_steps + k) * E + j] = 2.0 * acc;
            }
    rc = 0;
done:
    free(s1);
    free(s2);
    free(sw);
    return rc;
}

/* Element means of the exact Neumann datum w_r = alpha du/dn_x (the L2
 * projection into piecewise constants, whose error is the best-approximation
 * reference of Table dirconv's "projected" column), same rule as above. */
int orc_project_neumann(const double *nodes, int64_t n_nodes,
                        const int32_t *tris, int64_t E, double alpha, double T,
                        int32_t n_steps, const double *sources, int32_t n_src,
                        int32_t nrhs, int32_t q_space, int32_t n_time,
                        double *wproj)
{
    if (E < 1 || n_steps < 1 || nrhs < 1 || n_src < 1 || q_space < 1 ||
        q_space > 32 || n_time < 1 || n_time > 64)
        return -1;
    int nq = q_space * q_space;
    double *s1 = malloc(sizeof(double) * nq), *s2 = malloc(sizeof(double) * nq);
    double *sw = malloc(sizeof(double) * nq), tx[64], tw[64];
    double *area = malloc(sizeof(double) * E), *normal = malloc(sizeof(double) * 3 * E);
    int rc = -1;
    if (orc_triangle_rule(q_space, s1, s2, sw) || orc_gauss_legendre01(n_time, tx, tw) ||
        orc_triangle_geometry(nodes, n_nodes, tris, E, area, normal))
        goto done;
    double h = T / n_steps;
    for (int r = 0; r < nrhs; ++r)
        for (int k = 0; k < n_steps; ++k)
            for (int64_t j = 0; j < E; ++j) {
                const int32_t *t3 = tris + 3 * j;
                double acc = 0.0;
                for (int a = 0; a < nq; ++a) {
                    double x[3];
                    chi_plain(nodes + 3 * t3[0], nodes + 3 * t3[1], nodes + 3 * t3[2],
                              s1[a], s2[a], x);
                    for (int b = 0; b < n_time; ++b)
                        acc += sw[a] * tw[b] *
                               neumann_datum(sources + (int64_t)r * n_src * 5, n_src, alpha,
                                             x, normal + 3 * j, (k + tx[b]) * h);
                }
                wproj[((int64_t)r * n_steps + k) * E + j] = 2.0 * acc;
            }
    rc = 0;
done:
    free(s1);
    free(s2);
    free(sw);
    free(area);
    free(normal);
    return rc;
}

/* y_r^k = sum_{d=0}^{k} A^d x_r^{k-d}  (eq. V_mat layout), A: [n_steps][E][E]. */
int orc_toeplitz_matvec(const double *A, int64_t E, int32_t n_steps,
                        int32_t nrhs, const double *x, double *y)
{
    if (E < 1 || n_steps < 1 || nrhs < 1)
        return -1;
    for (int r = 0; r < nrhs; ++r)
        for (int k = 0; k < n_steps; ++k)
            for (int64_t l = 0; l < E; ++l) {
                double acc = 0.0;
                for (int d = 0; d <= k; ++d) {
                    const double *Arow = A + ((int64_t)d * E + l) * E;
                    const double *xv = x + ((int64_t)r * n_steps + (k - d)) * E;
                    for (int64_t j = 0; j < E; ++j)
                        acc += Arow[j] * xv[j];
                }
                y[((int64_t)r * n_steps + k) * E + l] = acc;
            }
    return 0;
}

/* f = (1/2 M_h + K_h) g with M_h = h diag(Delta) per time step. */
int orc_dirichlet_rhs(const double *area, const double *K, int64_t E,
                      double T, int32_t n_steps, int32_t nrhs,
                      const double *g, double *f)
{
    if (orc_toeplitz_matvec(K, E, n_steps, nrhs, g, f))
        return -1;
    double h = T / n_steps;
    for (int r = 0; r < nrhs; ++r)
        for (int k = 0; k < n_steps; ++k)
            for (int64_t l = 0; l < E; ++l) {
                int64_t i = ((int64_t)r * n_steps + k) * E + l;
                f[i] += 0.5 * h * area[l] * g[i];
            }
    return 0;
}

/* Block forward substitution (marching in time) for the lower-triangular
 * block-Toeplitz system of eq. V_mat:
 *   V^0 w^k = f^k - sum_{d=1}^{k} V^d w^{k-d},
 * with a plain dense Cholesky factorisation V^0 = L L^T.  Returns -5 if V^0
 * is not numerically positive definite. */
int orc_dirichlet_solve(const double *V, int64_t E, int32_t n_steps,
                        int32_t nrhs, const double *f, double *w)
{
    if (E < 1 || n_steps < 1 || nrhs < 1)
        return -1;
    double *L = malloc(sizeof(double) * E * E);
    double *rhs = malloc(sizeof(double) * E);
    int rc = 0;
    memcpy(L, V, sizeof(double) * E * E);
    for (int64_t c = 0; c < E && rc == 0; ++c) {
        double s = L[c * E + c];
        for (int64_t k = 0; k < c; ++k)
            s -= L[c * E + k] * L[c * E + k];
        if (!(s > 0.0)) {
            rc = -5;
            break;
        }
        double lcc = sqrt(s);
        L[c * E + c] = lcc;
        for (int64_t i = c + 1; i < E; ++i) {
            double t = L[i * E + c];
            for (int64_t k = 0; k < c; ++k)
                t -= L[i * E + k] * L[c * E + k];
            L[i * E + c] = t / lcc;
        }
    }
    for (int r = 0; r < nrhs && rc == 0; ++r)
        for (int k = 0; k < n_steps; ++k) {
            const double *fk = f + ((int64_t)r * n_steps + k) * E;
            double *wk = w + ((int64_t)r * n_steps + k) * E;
            for (int64_t l = 0; l < E; ++l) {
                double acc = fk[l];
                for (int d = 1; d <= k; ++d) {
                    const double *Vrow = V + ((int64_t)d * E + l) * E;
                    const double *wv = w + ((int64_t)r * n_steps + (k - d)) * E;
                    for (int64_t j = 0; j < E; ++j)
                        acc -= Vrow[j] * wv[j];
                }
                rhs[l] = acc;
            }
            for (int64_t i = 0; i < E; ++i) { /* L z = rhs */
                double t = rhs[i];
                for (int64_t k2 = 0; k2 < i; ++k2)
                    t -= L[i * E + k2] * rhs[k2];
                rhs[i] = t / L[i * E + i];
            }
            for (int64_t i = E - 1; i >= 0; --i) { /* L^T w = z */
                double t = rhs[i];
                for (int64_t k2 = i + 1; k2 < E; ++k2)
                    t -= L[k2 * E + i] * wk[k2];
                wk[i] = t / L[i * E + i];
            }
        }
    free(L);
    free(rhs);
    return rc;
}

/* err2 = sum_r || w_r - w_{h,r} ||^2_{L2(Sigma_h)}, ref2 = sum_r || w_r ||^2,
 * both by the same product rule as the projection (Sec. 6.1, error norm). */
int orc_neumann_error(const double *nodes, int64_t n_nodes,
                      const int32_t *tris, int64_t E, double alpha, double T,
                      int32_t n_steps, const double *sources, int32_t n_src,
                      int32_t nrhs, const double *w, int32_t q_space,
                      int32_t n_time, double *err2, double *ref2)
{
    if (E < 1 || n_steps < 1 || nrhs < 1 || q_space < 1 || q_space > 32 ||
        n_time < 1 || n_time > 64)
        return -1;
    int nq = q_space * q_space;
    double *s1 = malloc(sizeof(double) * nq), *s2 = malloc(sizeof(double) * nq);
    double *sw = malloc(sizeof(double) * nq), tx[64], tw[64];
    double *area = malloc(sizeof(double) * E), *normal = malloc(sizeof(double) * 3 * E);
    int rc = -1;
    if (orc_triangle_rule(q_space, s1, s2, sw) || orc_gauss_legendre01(n_time, tx, tw) ||
        orc_triangle_geometry(nodes, n_nodes, tris, E, area, normal))
        goto done;
    double h = T / n_steps, e2 = 0.0, r2 = 0.0;
    for (int r = 0; r < nrhs; ++r)
        for (int k = 0; k < n_steps; ++k)
            for (int64_t j = 0; j < E; ++j) {
                const int32_t *t3 = tris + 3 * j;
                double wh = w[((int64_t)r * n_steps + k) * E + j];
                double ae = 0.0, ar = 0.0;
                for (int a = 0; a < nq; ++a) {
                    double x[3];
                    chi_plain(nodes + 3 * t3[0], nodes + 3 * t3[1], nodes + 3 * t3[2],
                              s1[a], s2[a], x);
                    for (int b = 0; b < n_time; ++b) {
                        double we = neumann_datum(sources + (int64_t)r * n_src * 5, n_src,
                                                  alpha, x, normal + 3 * j, (k + tx[b]) * h);
                        ae += sw[a] * tw[b] * (we - wh) * (we - wh);
                        ar += sw[a] * tw[b] * we * we;
                    }
                }
                e2 += 2.0 * area[j] * h * ae;
                r2 += 2.0 * area[j] * h * ar;
            }
    *err2 = e2;
    *ref2 = r2;
    rc = 0;
done:
    free(s1);
    free(s2);
    free(sw);
    free(area);
    free(normal);
    return rc;
}

/* ---- piecewise-linear Dirichlet data (Sec. 3.2, Sec. 3.4) ------------------ */

/* Dense Cholesky of the SPD matrix A (n x n, overwritten by L, lower part);
 * -5 if a pivot is not positive. */
static int cholesky(double *A, int64_t n)
{
    for (int64_t c = 0; c < n; ++c) {
        double s = A[c * n + c];
        for (int64_t k = 0; k < c; ++k)
            s -= A[c * n + k] * A[c * n + k];
        if (!(s > 0.0))
            return -5;
        double lcc = sqrt(s);
        A[c * n + c] = lcc;
        for (int64_t i = c + 1; i < n; ++i) {
            double t = A[i * n + c];
            for (int64_t k = 0; k < c; ++k)
                t -= A[i * n + k] * A[c * n + k];
            A[i * n + c] = t / lcc;
        }
    }
    return 0;
}

static void cholesky_solve(const double *L, int64_t n, double *x)
{
    for (int64_t i = 0; i < n; ++i) {
        double t = x[i];
        for (int64_t k = 0; k < i; ++k)
            t -= L[i * n + k] * x[k];
        x[i] = t / L[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {
        double t = x[i];
        for (int64_t k = i + 1; k < n; ++k)
            t -= L[k * n + i] * x[k];
        x[i] = t / L[i * n + i];
    }
}

/* L2(Sigma_h) projection of g into X_h^{1,0} (piecewise linear in space,
 * piecewise constant in time): per step k the nodal vector g1^k solves
 *   M1 g1^k = b^k,  M1[i][m] = int_Gamma phi_i phi_m,
 *   b^k[i] = h^{-1} int_{t_k}^{t_{k+1}} int_Gamma g phi_i,
 * M1 from its exact element values Delta/12 (1 + delta_im), b^k by the
 * q_space conical rule and n_time Gauss points per step.
 * g1: [nrhs][n_steps][n_nodes]. */
int orc_project_dirichlet_p1(const double *nodes, int64_t n_nodes,
                             const int32_t *tris, int64_t E, double alpha,
                             double T, int32_t n_steps, const double *sources,
                             int32_t n_src, int32_t nrhs, int32_t q_space,
                             int32_t n_time, double *g1)
{
    if (E < 1 || n_nodes < 3 || n_steps < 1 || nrhs < 1 || n_src < 1 || q_space < 1 ||
        q_space > 32 || n_time < 1 || n_time > 64)
        return -1;
    int nq = q_space * q_space;
    double *s1 = malloc(sizeof(double) * nq), *s2 = malloc(sizeof(double) * nq);
    double *sw = malloc(sizeof(double) * nq), tx[64], tw[64];
    double *area = malloc(sizeof(double) * E), *normal = malloc(sizeof(double) * 3 * E);
    double *M = calloc((size_t)n_nodes * n_nodes, sizeof(double));
    int rc = -1;
    if (orc_triangle_rule(q_space, s1, s2, sw) || orc_gauss_legendre01(n_time, tx, tw) ||
        orc_triangle_geometry(nodes, n_nodes, tris, E, area, normal))
        goto done;
    for (int64_t j = 0; j < E; ++j)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                M[(int64_t)tris[3 * j + a] * n_nodes + tris[3 * j + b]] +=
                    area[j] / 12.0 * (a == b ? 2.0 : 1.0);
    if ((rc = cholesky(M, n_nodes)) != 0)
        goto done;
    rc = -1;
    double h = T / n_steps;
    for (int r = 0; r < nrhs; ++r)
        for (int k = 0; k < n_steps; ++k) {
            double *bk = g1 + ((int64_t)r * n_steps + k) * n_nodes;
            memset(bk, 0, sizeof(double) * n_nodes);
            for (int64_t j = 0; j < E; ++j) {
                const int32_t *t3 = tris + 3 * j;
                for (int a = 0; a < nq; ++a) {
                    double x[3], lam[3] = {1.0 - s1[a], s1[a] - s2[a], s2[a]};
                    chi_plain(nodes + 3 * t3[0], nodes + 3 * t3[1], nodes + 3 * t3[2],
                              s1[a], s2[a], x);
                    double acc = 0.0;
                    for (int b = 0; b < n_time; ++b)
                        acc += tw[b] * dirichlet_datum(sources + (int64_t)r * n_src * 5, n_src,
                                                       alpha, x, (k + tx[b]) * h);
                    /* (2 Delta sw) in space, (h tw) / h in time */
                    for (int v = 0; v < 3; ++v)
                        bk[t3[v]] += 2.0 * area[j] * sw[a] * lam[v] * acc;
                }
            }
            cholesky_solve(M, n_nodes, bk);
        }
    rc = 0;
done:
    free(s1);
    free(s2);
    free(sw);
    free(area);
    free(normal);
    free(M);
    return rc;
}

/* y_r^k = sum_{d=0}^{k} A^d x_r^{k-d} with rectangular blocks A^d [E][N]:
 * A [n_steps][E][N], x [nrhs][n_steps][N], y [nrhs][n_steps][E]. */
int orc_toeplitz_matvec_rect(const double *A, int64_t E, int64_t N, int32_t n_steps,
                             int32_t nrhs, const double *x, double *y)
{
    if (E < 1 || N < 1 || n_steps < 1 || nrhs < 1)
        return -1;
    for (int r = 0; r < nrhs; ++r)
        for (int k = 0; k < n_steps; ++k)
            for (int64_t l = 0; l < E; ++l) {
                double acc = 0.0;
                for (int d = 0; d <= k; ++d) {
                    const double *Arow = A + ((int64_t)d * E + l) * N;
                    const double *xv = x + ((int64_t)r * n_steps + (k - d)) * N;
                    for (int64_t i = 0; i < N; ++i)
                        acc += Arow[i] * xv[i];
                }
                y[((int64_t)r * n_steps + k) * E + l] = acc;
            }
    return 0;
}

/* f = (1/2 M_h + K_h) g1 with the p0 x p1 mass M_h = h blockdiag(M01),
 * M01[l][i] = int_{gamma_l} phi_i = Delta_l / 3 for the nodes i of l
 * (Sec. 3.4), and K_h the piecewise-linear double layer K1 [n_steps][E][N]. */
int orc_dirichlet_rhs_p1(const double *area, const int32_t *tris, const double *K1,
                         int64_t E, int64_t N, double T, int32_t n_steps, int32_t nrhs,
                         const double *g1, double *f)
{
    if (orc_toeplitz_matvec_rect(K1, E, N, n_steps, nrhs, g1, f))
        return -1;
    double h = T / n_steps;
    for (int r = 0; r < nrhs; ++r)
        for (int k = 0; k < n_steps; ++k)
            for (int64_t l = 0; l < E; ++l) {
                const double *gk = g1 + ((int64_t)r * n_steps + k) * N;
                double m = 0.0;
                for (int v = 0; v < 3; ++v)
                    m += gk[tris[3 * l + v]];
                f[((int64_t)r * n_steps + k) * E + l] += 0.5 * h * area[l] / 3.0 * m;
            }
    return 0;
}

/* ---- Neumann problem (Sec. 3.4) -------------------------------------------
 * Right-hand side of D_h u = (1/2 M_h^{T_x} - K_h^{T_x}) h with h in X_h^{0,0}
 * ([nrhs][n_steps][E]), K1 [n_steps][E][N] the piecewise-linear double layer
 * and M_h^{T_x} the blockwise transpose of the p0 x p1 mass:
 *   f_k[i] = (h_t / 2) sum_{l : i in l} Delta_l / 3 h_{k,l}
 *            - sum_{d=0}^{k} sum_l K1^d[l][i] h_{k-d,l},
 * f [nrhs][n_steps][N].                                                     */
int orc_neumann_rhs(const double *area, const int32_t *tris, const double *K1, int64_t E,
                    int64_t N, double T, int32_t n_steps, int32_t nrhs, const double *hd,
                    double *f)
{
    if (E < 1 || N < 1 || n_steps < 1 || nrhs < 1)
        return -1;
    double ht = T / n_steps;
    for (int r = 0; r < nrhs; ++r)
        for (int k = 0; k < n_steps; ++k) {
            double *fk = f + ((int64_t)r * n_steps + k) * N;
            for (int64_t i = 0; i < N; ++i)
                fk[i] = 0.0;
            const double *hk = hd + ((int64_t)r * n_steps + k) * E;
            for (int64_t l = 0; l < E; ++l)
                for (int v = 0; v < 3; ++v)
                    fk[tris[3 * l + v]] += 0.5 * ht * area[l] / 3.0 * hk[l];
            for (int d = 0; d <= k; ++d) {
                const double *Kd = K1 + (int64_t)d * E * N;
                const double *hv = hd + ((int64_t)r * n_steps + (k - d)) * E;
                for (int64_t l = 0; l < E; ++l)
                    for (int64_t i = 0; i < N; ++i)
                        fk[i] -= Kd[l * N + i] * hv[l];
            }
        }
    return 0;
}

/* Error of piecewise-linear Dirichlet data u1 [nrhs][n_steps][N] against the
 * exterior-source datum g (Sec. 6.1): err2 = sum_r ||g_r - u_h,r||^2 and
 * ref2 = sum_r ||g_r||^2 in L2(Sigma_h), u_h(x, t) = sum_v lambda_v(x)
 * u1_{k, node v} on step k, by the q_space x q_space conical rule and n_time
 * Gauss points per step.                                                    */
int orc_dirichlet_error_p1(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t E,
                           double alpha, double T, int32_t n_steps, const double *sources,
                           int32_t n_src, int32_t nrhs, const double *u1, int32_t q_space,
                           int32_t n_time, double *err2, double *ref2)
{
    if (E < 1 || n_steps < 1 || nrhs < 1 || q_space < 1 || q_space > 32 || n_time < 1 ||
        n_time > 64)
        return -1;
    int nq = q_space * q_space;
    double *s1 = malloc(sizeof(double) * nq), *s2 = malloc(sizeof(double) * nq);
    double *sw = malloc(sizeof(double) * nq), tx[64], tw[64];
    double *area = malloc(sizeof(double) * E), *normal = malloc(sizeof(double) * 3 * E);
    int rc = -1;
    if (orc_triangle_rule(q_space, s1, s2, sw) || orc_gauss_legendre01(n_time, tx, tw) ||
        orc_triangle_geometry(nodes, n_nodes, tris, E, area, normal))
        goto done;
    double h = T / n_steps, e2 = 0.0, r2 = 0.0;
    for (int r = 0; r < nrhs; ++r)
        for (int k = 0; k < n_steps; ++k)
            for (int64_t j = 0; j < E; ++j) {
                const int32_t *t3 = tris + 3 * j;
                const double *uk = u1 + ((int64_t)r * n_steps + k) * n_nodes;
                double ae = 0.0, ar = 0.0;
                for (int a = 0; a < nq; ++a) {
                    double x[3];
                    chi_plain(nodes + 3 * t3[0], nodes + 3 * t3[1], nodes + 3 * t3[2],
                              s1[a], s2[a], x);
                    double uh = (1.0 - s1[a]) * uk[t3[0]] + (s1[a] - s2[a]) * uk[t3[1]] +
                                s2[a] * uk[t3[2]];
                    for (int b = 0; b < n_time; ++b) {
                        double g = dirichlet_datum(sources + (int64_t)r * n_src * 5, n_src, alpha,
                                                   x, (k + tx[b]) * h);
                        ae += sw[a] * tw[b] * (g - uh) * (g - uh);
                        ar += sw[a] * tw[b] * g * g;
                    }
                }
                e2 += 2.0 * area[j] * h * ae;
                r2 += 2.0 * area[j] * h * ar;
            }
    *err2 = e2;
    *ref2 = r2;
    rc = 0;
done:
    free(s1);
    free(s2);
    free(sw);
    free(area);
    free(normal);
    return rc;
}

/* ---- non-uniform time grids ----------------------------------------------
 * Blocks packed at b(k,i) = k(k+1)/2 + i (k >= i), times [n_steps + 1],
 * vectors [nrhs][n_steps][E].                                               */

/* y^k = sum_{i <= k} A^{k,i} x^i */
int orc_matvec_nu(const double *A, int64_t E, int32_t n_steps, int32_t nrhs, const double *x,
                  double *y)
{
    if (E < 1 || n_steps < 1 || nrhs < 1)
        return -1;
    for (int r = 0; r < nrhs; ++r)
        for (int k = 0; k < n_steps; ++k)
            for (int64_t l = 0; l < E; ++l) {
                double acc = 0.0;
                for (int i = 0; i <= k; ++i) {
                    const double *row = A + (((int64_t)k * (k + 1) / 2 + i) * E + l) * E;
                    const double *xv = x + ((int64_t)r * n_steps + i) * E;
                    for (int64_t j = 0; j < E; ++j)
                        acc += row[j] * xv[j];
                }
                y[((int64_t)r * n_steps + k) * E + l] = acc;
            }
    return 0;
}

/* Block forward substitution: w^k = (V^{k,k})^{-1} (f^k - sum_{i<k} V^{k,i} w^i),
 * each diagonal block by its own dense Cholesky factorisation. */
int orc_solve_nu(const double *V, int64_t E, int32_t n_steps, int32_t nrhs, const double *f,
                 double *w)
{
    if (E < 1 || n_steps < 1 || nrhs < 1)
        return -1;
    double *L = malloc(sizeof(double) * E * E);
    double *rhs = malloc(sizeof(double) * E);
    int rc = 0;
    for (int k = 0; k < n_steps && rc == 0; ++k) {
        memcpy(L, V + ((int64_t)k * (k + 1) / 2 + k) * E * E, sizeof(double) * E * E);
        if ((rc = cholesky(L, E)) != 0)
            break;
        for (int r = 0; r < nrhs; ++r) {
            const double *fk = f + ((int64_t)r * n_steps + k) * E;
            for (int64_t l = 0; l < E; ++l) {
                double acc = fk[l];
                for (int i = 0; i < k; ++i) {
                    const double *row = V + (((int64_t)k * (k + 1) / 2 + i) * E + l) * E;
                    const double *wv = w + ((int64_t)r * n_steps + i) * E;
                    for (int64_t j = 0; j < E; ++j)
                        acc -= row[j] * wv[j];
                }
                rhs[l] = acc;
            }
            cholesky_solve(L, E, rhs);
            memcpy(w + ((int64_t)r * n_steps + k) * E, rhs, sizeof(double) * E);
        }
    }
    free(L);
    free(rhs);
    return rc;
}

/* Element means of the Dirichlet datum over [t_k, t_{k+1}] x gamma_j. */
int orc_project_dirichlet_nu(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t E,
                             double alpha, const double *times, int32_t n_steps,
                             const double *sources, int32_t n_src, int32_t nrhs, int32_t q_space,
                             int32_t n_time, double *g)
{
    if (E < 1 || n_steps < 1 || nrhs < 1 || n_src < 1 || q_space < 1 || q_space > 32 ||
        n_time < 1 || n_time > 64)
        return -1;
    int nq = q_space * q_space;
    double *s1 = malloc(sizeof(double) * nq), *s2 = malloc(sizeof(double) * nq);
    double *sw = malloc(sizeof(double) * nq), tx[64], tw[64];
    int rc = -1;
    if (orc_triangle_rule(q_space, s1, s2, sw) || orc_gauss_legendre01(n_time, tx, tw))
        goto done;
    for (int r = 0; r < nrhs; ++r)
        for (int k = 0; k < n_steps; ++k) {
            const double t0 = times[k], hk = times[k + 1] - times[k];
            for (int64_t j = 0; j < E; ++j) {
                const int32_t *t3 = tris + 3 * j;
                double acc = 0.0;
                for (int a = 0; a < nq; ++a) {
                    double x[3];
                    chi_plain(nodes + 3 * t3[0], nodes + 3 * t3[1], nodes + 3 * t3[2], s1[a],
                              s2[a], x);
                    for (int b = 0; b < n_time; ++b)
                        acc += sw[a] * tw[b] *
                               dirichlet_datum(sources + (int64_t)r * n_src * 5, n_src, alpha, x,
                                               t0 + tx[b] * hk);
                }
                g[((int64_t)r * n_steps + k) * E + j] = 2.0 * acc;
            }
        }
    rc = 0;
done:
    free(s1);
    free(s2);
    free(sw);
    return rc;
}

/* f^k = (h_k / 2) Delta g^k + sum_{i <= k} K^{k,i} g^i */
int orc_dirichlet_rhs_nu(const double *area, const double *K, int64_t E, const double *times,
                         int32_t n_steps, int32_t nrhs, const double *g, double *f)
{
    if (orc_matvec_nu(K, E, n_steps, nrhs, g, f))
        return -1;
    for (int r = 0; r < nrhs; ++r)
        for (int k = 0; k < n_steps; ++k)
            for (int64_t l = 0; l < E; ++l) {
                int64_t idx = ((int64_t)r * n_steps + k) * E + l;
                f[idx] += 0.5 * (times[k + 1] - times[k]) * area[l] * g[idx];
            }
    return 0;
}

/* L2(Sigma_h) error of piecewise-constant w against the Neumann datum. */
int orc_neumann_error_nu(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t E,
                         double alpha, const double *times, int32_t n_steps,
                         const double *sources, int32_t n_src, int32_t nrhs, const double *w,
                         int32_t q_space, int32_t n_time, double *err2, double *ref2)
{
    if (E < 1 || n_steps < 1 || nrhs < 1 || q_space < 1 || q_space > 32 || n_time < 1 ||
        n_time > 64)
        return -1;
    int nq = q_space * q_space;
    double *s1 = malloc(sizeof(double) * nq), *s2 = malloc(sizeof(double) * nq);
    double *sw = malloc(sizeof(double) * nq), tx[64], tw[64];
    double *area = malloc(sizeof(double) * E), *normal = malloc(sizeof(double) * 3 * E);
    int rc = -1;
    if (orc_triangle_rule(q_space, s1, s2, sw) || orc_gauss_legendre01(n_time, tx, tw) ||
        orc_triangle_geometry(nodes, n_nodes, tris, E, area, normal))
        goto done;
    double e2 = 0.0, r2 = 0.0;
    for (int r = 0; r < nrhs; ++r)
        for (int k = 0; k < n_steps; ++k) {
            const double t0 = times[k], hk = times[k + 1] - times[k];
            for (int64_t j = 0; j < E; ++j) {
                const int32_t *t3 = tris + 3 * j;
                double wh = w[((int64_t)r * n_steps + k) * E + j];
                double ae = 0.0, ar = 0.0;
                for (int a = 0; a < nq; ++a) {
                    double x[3];
                    chi_plain(nodes + 3 * t3[0], nodes + 3 * t3[1], nodes + 3 * t3[2], s1[a],
                              s2[a], x);
                    for (int b = 0; b < n_time; ++b) {
                        double we = neumann_datum(sources + (int64_t)r * n_src * 5, n_src, alpha,
                                                  x, normal + 3 * j, t0 + tx[b] * hk);
                        ae += sw[a] * tw[b] * (we - wh) * (we - wh);
                        ar += sw[a] * tw[b] * we * we;
                    }
                }
                e2 += 2.0 * area[j] * hk * ae;
                r2 += 2.0 * area[j] * hk * ar;
            }
        }
    *err2 = e2;
    *ref2 = r2;
    rc = 0;
done:
    free(s1);
    free(s2);
    free(sw);
    free(area);
    free(normal);
    return rc;
}
