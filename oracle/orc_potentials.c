/*
 * orc_potentials.c -- the discretised representation formula (eq. repr):
 * single-layer potential V~ w_h and double-layer potential W u_h at points
 * (x, t) off the boundary (Sec. 3.5, "Single- and double-layer potential").
 * TEST INFRASTRUCTURE ONLY; see orc.h.
 *
 * With t = t_k + eps, t_k = k h, eps in [0, h] (k = min(floor(t/h), E_t - 1),
 * so that t = T uses the last step with eps = h), the potentials are the
 * paper's sums over the past steps d = 0..k-1 of the coefficient of step k-d
 * (1-based) times the difference of the temporal antiderivative at d h + eps
 * and (d+1) h + eps, plus the coefficient of step k+1 times the difference
 * at 0 and eps:
 *   V~ w_h(x,t) = sum_j int_{gamma_j} { sum_d w_{k-d,j} [G^{dtau}(x-y, dh+eps)
 *                   - G^{dtau}(x-y, (d+1)h+eps)]
 *                 + w_{k+1,j} [G^{dtau}(x-y, 0) - G^{dtau}(x-y, eps)] } ds_y,
 *   W u_h(x,t)  = the same with u_h in X_h^{1,0} (nodal hat functions in
 *                 space) and alpha dG^{dtau}/dn_y (eq. dn_G_dtau) in place of
 *                 G^{dtau} (eq. G_dtau); the delta = 0 values are the limits
 *                 of eq. G_dtau_lim_d and eq. dn_G_dtau_lim_r.
 * The points are off Gamma_h, so every integrand is smooth: each triangle
 * is integrated by the q x q conical rule, the antiderivatives in time are
 * exact.  Arrays: w [nrhs][n_steps][E] (0-based step index = 1-based - 1),
 * u1 [nrhs][n_steps][n_nodes], points [n_pts][4] = (x1, x2, x3, t),
 * slp, dlp [nrhs][n_pts].
 */
#include <math.h>
#include <stdlib.h>
#include "orc.h"

/* step index and offset of a time in [0, T] (the convention above) */
static void step_of(double t, double h, int32_t n_steps, int *k, double *eps)
{
    int kk = (int)floor(t / h);
    if (kk > n_steps - 1)
        kk = n_steps - 1;
    if (kk < 0)
        kk = 0;
    *k = kk;
    *eps = t - kk * h;
}

int orc_potentials(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t E,
                   double alpha, double T, int32_t n_steps, const double *w, const double *u1,
                   int32_t nrhs, const double *points, int64_t n_pts, int32_t q,
                   double *slp, double *dlp)
{
    if (E < 1 || n_nodes < 3 || n_steps < 1 || nrhs < 1 || n_pts < 1 || q < 1 || q > 32 ||
        !(alpha > 0) || !(T > 0))
        return -1;
    if ((slp && !w) || (dlp && !u1))
        return -1;
    for (int64_t p = 0; p < n_pts; ++p)
        if (!(points[4 * p + 3] >= 0.0 && points[4 * p + 3] <= T))
            return -1;
    const int nq = q * q;
    double *s1 = malloc(sizeof(double) * nq), *s2 = malloc(sizeof(double) * nq);
    double *sw = malloc(sizeof(double) * nq);
    double *area = malloc(sizeof(double) * E), *normal = malloc(sizeof(double) * 3 * E);
    int rc = -1;
    if (!s1 || !s2 || !sw || !area || !normal)
        goto done;
    if (orc_triangle_rule(q, s1, s2, sw) ||
        orc_triangle_geometry(nodes, n_nodes, tris, E, area, normal))
        goto done;
    const double h = T / n_steps;
    for (int r = 0; r < nrhs; ++r)
        for (int64_t p = 0; p < n_pts; ++p) {
            const double *x = points + 4 * p;
            int k;
            double eps;
            step_of(x[3], h, n_steps, &k, &eps);
            double vs = 0.0, ws = 0.0;
            for (int64_t j = 0; j < E; ++j) {
                const int32_t *t3 = tris + 3 * j;
                const double *P0 = nodes + 3 * t3[0], *P1 = nodes + 3 * t3[1],
                             *P2 = nodes + 3 * t3[2];
                const double *n = normal + 3 * j;
                for (int a = 0; a < nq; ++a) {
                    double y[3], rv[3];
                    for (int c = 0; c < 3; ++c) {
                        y[c] = P0[c] + s1[a] * (P1[c] - P0[c]) + s2[a] * (P2[c] - P1[c]);
                        rv[c] = x[c] - y[c];
                    }
                    const double rho = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
                    const double rn = rv[0] * n[0] + rv[1] * n[1] + rv[2] * n[2];
                    const double lam[3] = {1.0 - s1[a], s1[a] - s2[a], s2[a]};
                    const double wq = 2.0 * area[j] * sw[a];
                    /* past steps i = k-d (1-based), i.e. 0-based index k-1-d */
                    for (int d = 0; d <= k - 1; ++d) {
                        const int i0 = k - 1 - d;
                        if (slp) {
                            double c = w[((int64_t)r * n_steps + i0) * E + j];
                            vs += wq * c *
                                  (orc_G_dtau(rho, d * h + eps, alpha) -
                                   orc_G_dtau(rho, (d + 1) * h + eps, alpha));
                        }
                        if (dlp) {
                            double c = 0.0;
                            for (int v = 0; v < 3; ++v)
                                c += lam[v] * u1[((int64_t)r * n_steps + i0) * n_nodes + t3[v]];
                            ws += wq * c *
                                  (orc_dn_G_dtau(rn, rho, d * h + eps, alpha) -
                                   orc_dn_G_dtau(rn, rho, (d + 1) * h + eps, alpha));
                        }
                    }
                    /* the current step k+1 (1-based), 0-based index k, on [t_k, t] */
                    if (slp) {
                        double c = w[((int64_t)r * n_steps + k) * E + j];
                        vs += wq * c * (orc_G_dtau(rho, 0.0, alpha) - orc_G_dtau(rho, eps, alpha));
                    }
                    if (dlp) {
                        double c = 0.0;
                        for (int v = 0; v < 3; ++v)
                            c += lam[v] * u1[((int64_t)r * n_steps + k) * n_nodes + t3[v]];
                        ws += wq * c *
                              (orc_dn_G_dtau(rn, rho, 0.0, alpha) - orc_dn_G_dtau(rn, rho, eps, alpha));
                    }
                }
            }
            if (slp)
                slp[(int64_t)r * n_pts + p] = vs;
            if (dlp)
                dlp[(int64_t)r * n_pts + p] = ws;
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
