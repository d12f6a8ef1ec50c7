/*
 * orc_quad.c -- quadrature rules of the oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Reference triangle  T = { (s1, s2) : 0 <= s2 <= s1 <= 1 },  |T| = 1/2,
 * mapped to a flat triangle (P0, P1, P2) by
 *     chi(s) = P0 + s1 (P1 - P0) + s2 (P2 - P1),   |det| = 2 Delta,
 * so that a pair integral is 4 Delta_l Delta_j times an integral over T x T
 * (eq. quad_reg).
 *
 * Regular rule (eq. st): Stroud conical product on T, s1 = sigma1,
 * s2 = sigma1 sigma2, Gauss-Jacobi (weight sigma1) in sigma1 and
 * Gauss-Legendre in sigma2, q points each (exact to degree 2q-1).
 *
 * Regularised rules for touching pairs (eq. quad_duffy, eq. ss): the paper
 * cites Duffy/Sauter-Schwab substitutions without printing the maps F^s and
 * Jacobians J^s.  The maps below are this project's own derivation of the
 * same idea (collect the singular set at one variable zeta of [0,1]^4 whose
 * power in the Jacobian cancels the kernel singularity), each a tensor
 * Gauss-Legendre rule with m points per direction:
 *   identical pair: 6 sub-domains, Jacobian zeta (1-zeta)^2 sigma1
 *   common edge   : 4 sub-domains, Jacobian zeta^2 (1-zeta) [* a]
 *   common vertex : 2 sub-domains, Jacobian zeta^3 a
 * (derivations in orc_ss_rule below).
 */
#include <math.h>
#include <stdlib.h>
#include "orc.h"

/* Legendre P_n(y) and P_{n-1}(y) by the three-term recurrence. */
static void legendre_pair(int n, double y, double *pn, double *pnm1)
{
    double p0 = 1.0, p1 = y;
    if (n == 0) {
        *pn = 1.0;
        *pnm1 = 0.0;
        return;
    }
    for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * y * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *pnm1 = p0;
}

static double legendre(int n, double y)
{
    double a, b;
    legendre_pair(n, y, &a, &b);
    return a;
}

/* f(y) = P_n(y) (kind 0) or P_n(y) + P_{n+1}(y) (kind 1). */
static double root_fn(int kind, int n, double y)
{
    return kind == 0 ? legendre(n, y) : legendre(n, y) + legendre(n + 1, y);
}

/* All n roots of root_fn in (-1, 1), ascending: sign changes on a fine grid,
 * each refined by bisection to adjacent doubles.  For kind 1 the root at
 * y = -1 is excluded by starting the grid just inside the interval. */
static int roots(int kind, int n, double *y)
{
    int grid = 4000 * (n + 1), found = 0;
    double a = -1.0 + 1e-12, fa = root_fn(kind, n, a);
    for (int g = 1; g <= grid && found < n; ++g) {
        double b = (g == grid) ? 1.0 - 1e-12 : -1.0 + 2.0 * g / grid;
        double fb = root_fn(kind, n, b);
        if (fa == 0.0) {
            y[found++] = a;
        } else if (fa * fb < 0.0) {
            double lo = a, hi = b, flo = fa;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi);
                if (mid <= lo || mid >= hi)
                    break;
                double fm = root_fn(kind, n, mid);
                if (fm == 0.0) {
                    lo = hi = mid;
                    break;
                }
                if (flo * fm < 0.0) {
                    hi = mid;
                } else {
                    lo = mid;
                    flo = fm;
                }
            }
            y[found++] = 0.5 * (lo + hi);
        }
        a = b;
        fa = fb;
    }
    return found == n ? 0 : -1;
}

/* n-point Gauss-Legendre rule on [0,1]:  w = 2 / ((1 - y^2) P_n'(y)^2) on
 * [-1, 1], halved for [0, 1], with (1 - y^2) P_n' = n (P_{n-1} - y P_n); the
 * y P_n term (zero at an exact root) removes the first-order effect of the
 * last-bit error of the computed node. */
int orc_gauss_legendre01(int n, double *x, double *w)
{
    if (n < 1 || n > 64)
        return -1;
    double *y = (double *)malloc(sizeof(double) * n);
    if (roots(0, n, y)) {
        free(y);
        return -1;
    }
    for (int i = 0; i < n; ++i) {
        double pn, pnm1;
        legendre_pair(n, y[i], &pn, &pnm1);
        double one_m_y2 = (1.0 - y[i]) * (1.0 + y[i]);
        double dp = n * (pnm1 - y[i] * pn);
        double wy = 2.0 * one_m_y2 / (dp * dp);
        x[i] = 0.5 * (1.0 + y[i]);
        w[i] = 0.5 * wy;
    }
    free(y);
    return 0;
}

/* n-point Gauss rule for the weight x on [0,1] (Gauss-Jacobi with
 * (alpha, beta) = (0, 1) after y = 2x - 1).  Its nodes are the interior nodes
 * of the (n+1)-point Gauss-Radau rule anchored at y = -1, i.e. the roots of
 * (P_n + P_{n+1})(y) / (1 + y), and its weights are the Radau weights
 * (1 - y) / ((n+1) P_n(y))^2 times (1 + y); the map to [0,1] divides by 4. */
int orc_gauss_jacobi01(int n, double *x, double *w)
{
    if (n < 1 || n > 64)
        return -1;
    double *y = (double *)malloc(sizeof(double) * n);
    if (roots(1, n, y)) {
        free(y);
        return -1;
    }
    for (int i = 0; i < n; ++i) {
        double pn = legendre(n, y[i]);
        double wy = (1.0 - y[i]) * (1.0 + y[i]) / (((n + 1) * pn) * ((n + 1) * pn));
        x[i] = 0.5 * (1.0 + y[i]);
        w[i] = 0.25 * wy;
    }
    free(y);
    return 0;
}

/* Conical product rule on T with q*q points; weights sum to |T| = 1/2. */
int orc_triangle_rule(int q, double *s1, double *s2, double *w)
{
    if (q < 1 || q > 32)
        return -1;
    double xj[32], wj[32], xl[32], wl[32];
    if (orc_gauss_jacobi01(q, xj, wj) || orc_gauss_legendre01(q, xl, wl))
        return -1;
    for (int a = 0; a < q; ++a)
        for (int b = 0; b < q; ++b) {
            int k = a * q + b;
            s1[k] = xj[a];
            s2[k] = xj[a] * xl[b];
            w[k] = wj[a] * wl[b];
        }
    return 0;
}

int orc_ss_rule_size(int cls, int m)
{
    int m4 = m * m * m * m;
    switch (cls) {
    case ORC_IDENTICAL: return 6 * m4;
    case ORC_EDGE: return 4 * m4;
    case ORC_VERTEX: return 2 * m4;
    default: return 0;
    }
}

/*
 * Regularised rule on T x T for a touching pair, returning points (s, t) and
 * weights so that  int_T int_T f(s, t) dt ds ~= sum_k w_k f(s_k, t_k).
 * Both triangles use chi; the caller orders their vertices so that the shared
 * vertices come first and in the same order (P0 common for a vertex pair,
 * P0 P1 common for an edge pair, same triangle for the identical pair).
 *
 * Identical pair.  With z = t - s, the set of s with s, s + z in T is the
 * copy of T scaled by L(z) = 1 - phi(z) and shifted to a corner c(z); the
 * sign pattern of (z1, z2, z1 - z2) splits z into six cones on which phi is
 * linear.  Writing z = zeta * (direction of the cone edge at phi = 1),
 * s = c(z) + (1 - zeta) stilde, stilde = (p1, p1 p2) in T, gives Jacobian
 * zeta (1 - zeta)^2 p1 on [0,1]^4 = (zeta, u, p1, p2).
 *
 * Edge pair (shared edge s2 = t2 = 0, s1 = t1).  With u = t1 - s1 the set of
 * admissible s1 for fixed (u, s2, t2) is an interval of length 1 - zeta where
 * zeta is u + s2, t2, s2 or t2 - u on four cones of (u, s2, t2); zeta and two
 * simplex coordinates parametrise the cone (Jacobian zeta^2 [* a]) and
 * s1 = lo + (1 - zeta) sigma.
 *
 * Vertex pair (shared vertex s = t = 0).  Duffy coordinates s = (S, S p2),
 * t = (R, R q2) and the split S >= R / S < R with the larger one = zeta and
 * the smaller = zeta a: Jacobian zeta^3 a.
 */
int orc_ss_rule(int cls, int m, double *s1, double *s2, double *t1, double *t2,
                double *w)
{
    if (m < 1 || m > 32)
        return -1;
    double g[32], gw[32];
    if (orc_gauss_legendre01(m, g, gw))
        return -1;
    int k = 0;
    if (cls == ORC_IDENTICAL) {
        for (int reg = 0; reg < 6; ++reg)
            for (int iz = 0; iz < m; ++iz)
                for (int iu = 0; iu < m; ++iu)
                    for (int i1 = 0; i1 < m; ++i1)
                        for (int i2 = 0; i2 < m; ++i2) {
                            double zt = g[iz], u = g[iu], p1 = g[i1], p2 = g[i2];
                            double z1, z2, c1, c2;
                            switch (reg) {
                            case 0: /* z1 >= z2 >= 0          */
                                z1 = zt; z2 = zt * u; c1 = 0.0; c2 = 0.0; break;
                            case 1: /* z2 > z1 >= 0           */
                                z1 = zt * u; z2 = zt; c1 = z2 - z1; c2 = 0.0; break;
                            case 2: /* z1 >= 0 > z2           */
                                z1 = zt * u; z2 = -zt * (1.0 - u); c1 = -z2; c2 = -z2; break;
                            case 3: /* z2 >= 0 > z1           */
                                z1 = -zt * u; z2 = zt * (1.0 - u); c1 = z2 - z1; c2 = 0.0; break;
                            case 4: /* 0 > z1 >= z2           */
                                z1 = -zt * u; z2 = -zt; c1 = -z2; c2 = -z2; break;
                            default: /* 0 > z2 > z1           */
                                z1 = -zt; z2 = -zt * u; c1 = -z1; c2 = -z2; break;
                            }
                            double L = 1.0 - zt;
                            s1[k] = c1 + L * p1;
                            s2[k] = c2 + L * p1 * p2;
                            t1[k] = s1[k] + z1;
                            t2[k] = s2[k] + z2;
                            w[k] = gw[iz] * gw[iu] * gw[i1] * gw[i2] * zt * L * L * p1;
                            ++k;
                        }
    } else if (cls == ORC_EDGE) {
        for (int reg = 0; reg < 4; ++reg)
            for (int iz = 0; iz < m; ++iz)
                for (int ia = 0; ia < m; ++ia)
                    for (int ib = 0; ib < m; ++ib)
                        for (int is = 0; is < m; ++is) {
                            double zt = g[iz], a = g[ia], b = g[ib], sg = g[is];
                            double L = 1.0 - zt, jac = gw[iz] * gw[ia] * gw[ib] * gw[is];
                            double S1, S2, T1, T2;
                            switch (reg) {
                            case 0: { /* u >= 0, t2 <= s2 + u : zeta = u + s2 */
                                double u = zt * a;
                                S2 = zt * (1.0 - a); T2 = zt * b;
                                S1 = S2 + L * sg; T1 = S1 + u;
                                jac *= zt * zt * L;
                                break;
                            }
                            case 1: { /* u >= 0, t2 > s2 + u : zeta = t2 */
                                double u = zt * a * b;
                                T2 = zt; S2 = zt * a * (1.0 - b);
                                S1 = T2 - u + L * sg; T1 = S1 + u;
                                jac *= zt * zt * L * a;
                                break;
                            }
                            case 2: { /* u < 0, s2 >= t2 - u : zeta = s2 */
                                double mneg = zt * a * b;
                                S2 = zt; T2 = zt * a * (1.0 - b);
                                S1 = zt + L * sg; T1 = S1 - mneg;
                                jac *= zt * zt * L * a;
                                break;
                            }
                            default: { /* u < 0, s2 < t2 - u : zeta = t2 - u */
                                double mneg = zt * a;
                                T2 = zt * (1.0 - a); S2 = zt * b;
                                S1 = zt + L * sg; T1 = S1 - mneg;
                                jac *= zt * zt * L;
                                break;
                            }
                            }
                            s1[k] = S1; s2[k] = S2; t1[k] = T1; t2[k] = T2; w[k] = jac;
                            ++k;
                        }
    } else if (cls == ORC_VERTEX) {
        for (int reg = 0; reg < 2; ++reg)
            for (int iz = 0; iz < m; ++iz)
                for (int ia = 0; ia < m; ++ia)
                    for (int ip = 0; ip < m; ++ip)
                        for (int iq = 0; iq < m; ++iq) {
                            double zt = g[iz], a = g[ia], p2 = g[ip], q2 = g[iq];
                            double S = reg == 0 ? zt : zt * a;
                            double R = reg == 0 ? zt * a : zt;
                            s1[k] = S; s2[k] = S * p2;
                            t1[k] = R; t2[k] = R * q2;
                            w[k] = gw[iz] * gw[ia] * gw[ip] * gw[iq] * zt * zt * zt * a;
                            ++k;
                        }
    } else {
        return -1;
    }
    return 0;
}
