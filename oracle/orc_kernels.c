/*
 * orc_kernels.c -- heat kernel, its scaled normal derivative and the closed
 * form temporal antiderivatives of the space-time heat BEM, written out
 * literally from the paper (TEST INFRASTRUCTURE ONLY; see orc.h).
 *
 * Notation: rho = ||r||, rn = r . n_y, x = rho / (2 sqrt(alpha delta)).
 */
#include <math.h>
#include "orc.h"

static const double PI = 3.14159265358979323846264338327950288;

/* Fundamental solution G_alpha(r, delta) (Sec. 2): zero for delta <= 0. */
double orc_heat_kernel(double rho, double delta, double alpha)
{
    if (delta <= 0.0)
        return 0.0;
    return pow(4.0 * PI * alpha * delta, -1.5) *
           exp(-rho * rho / (4.0 * alpha * delta));
}

/* Scaled normal derivative alpha dG_alpha/dn_y (Sec. 2). */
double orc_dn_heat_kernel(double rn, double rho, double delta, double alpha)
{
    if (delta <= 0.0)
        return 0.0;
    return rn / (16.0 * pow(PI * alpha, 1.5) * pow(delta, 2.5)) *
           exp(-rho * rho / (4.0 * alpha * delta));
}

/* G^{dtau}(r, delta), eq. G_dtau; delta -> 0+ limit eq. G_dtau_lim_d.
 * At rho = 0 (delta > 0) the continuous extension 1/(4 pi alpha sqrt(pi alpha
 * delta)) is returned (erf(x)/rho -> 1/sqrt(pi alpha delta)); the paper does
 * not need this value. */
double orc_G_dtau(double rho, double delta, double alpha)
{
    if (delta <= 0.0)
        return 1.0 / (4.0 * PI * alpha * rho);
    if (rho <= 0.0)
        return 1.0 / (4.0 * PI * alpha * sqrt(PI * alpha * delta));
    return erf(rho / (2.0 * sqrt(alpha * delta))) / (4.0 * PI * alpha * rho);
}

/* G^{dtau dt}(r, delta), eq. G_dtau_dt, with the two limits of Sec. 3.1
 * ("Stable evaluations of V^d"): delta -> 0+ gives rho/(8 pi alpha^2),
 * rho -> 0+ gives sqrt(delta)/(2 sqrt(pi^3 alpha^3)). */
double orc_G_dtau_dt(double rho, double delta, double alpha)
{
    if (delta <= 0.0)
        return rho / (8.0 * PI * alpha * alpha);
    if (rho <= 0.0)
        return sqrt(delta) / (2.0 * sqrt(PI * PI * PI * alpha * alpha * alpha));
    double x = rho / (2.0 * sqrt(alpha * delta));
    return (1.0 / (4.0 * PI)) *
           ((rho / (2.0 * alpha * alpha) + delta / (alpha * rho)) * erf(x) +
            sqrt(delta) / sqrt(PI * alpha * alpha * alpha) * exp(-x * x));
}

/* psi(x) = erf(x)/2 - erf(x)/(4x^2) + exp(-x^2)/(2 sqrt(pi) x): the bracket
 * of eq. dG after dividing by 1/alpha, i.e.
 *   alpha dG^{dtau dt}/dn_y = -(rn / (4 pi alpha rho)) psi(x).
 * psi_direct is the printed expression; psi_series is its Taylor series
 *   psi(x) = (2/sqrt(pi)) sum_m (-1)^m x^{2m+1} / (m! (2m+1) (2m+3)),
 * used below ORC_SERIES_X where the printed form cancels. */
double orc_psi_direct(double x)
{
    double e = erf(x);
    return 0.5 * e - e / (4.0 * x * x) + exp(-x * x) / (2.0 * sqrt(PI) * x);
}

double orc_psi_series(double x)
{
    double x2 = x * x, term = x, sum = 0.0; /* term = (-1)^m x^{2m+1} / m! */
    for (int m = 0; m < 40; ++m) {
        double c = term / ((2.0 * m + 1.0) * (2.0 * m + 3.0));
        sum += c;
        if (fabs(c) < 1e-18 * fabs(sum))
            break;
        term *= -x2 / (m + 1.0);
    }
    return 2.0 / sqrt(PI) * sum;
}

/* alpha dG^{dtau dt}/dn_y (r, delta), eq. dG, with the limits of Sec. 3.2
 * ("Stable evaluations of K^d"): delta -> 0+ gives -rn/(8 pi alpha rho),
 * rho -> 0+ gives 0. */
double orc_dn_G_dtau_dt(double rn, double rho, double delta, double alpha)
{
    if (delta <= 0.0)
        return -rn / (8.0 * PI * alpha * rho);
    if (rho <= 0.0)
        return 0.0;
    double x = rho / (2.0 * sqrt(alpha * delta));
    if (x < ORC_SERIES_X)
        return -rn / (4.0 * PI * alpha * rho) * orc_psi_series(x);
    return -(1.0 / (4.0 * PI)) * (rn / rho) *
           ((1.0 / (2.0 * alpha) - delta / (rho * rho)) * erf(x) +
            sqrt(delta) / (rho * sqrt(PI * alpha)) * exp(-x * x));
}

/* alpha dG^{dtau}/dn_y (r, delta), eq. dn_G_dtau; delta -> 0+ limit
 * eq. dn_G_dtau_lim_r = rn / (4 pi rho^3).  For small x the bracket
 * erf(x)/rho - exp(-x^2)/sqrt(pi alpha delta) = (erf(x) - 2x e^{-x^2}/sqrt(pi))/rho
 * is taken from its series (4/sqrt(pi)) sum_{m>=1} (-1)^{m+1} x^{2m+1} /
 * ((m-1)! (2m+1)).  The assembly only evaluates delta = 0. */
double orc_dn_G_dtau(double rn, double rho, double delta, double alpha)
{
    if (delta <= 0.0)
        return rn / (4.0 * PI * rho * rho * rho);
    if (rho <= 0.0)
        return 0.0;
    double x = rho / (2.0 * sqrt(alpha * delta));
    double bracket;
    if (x < ORC_SERIES_X) {
        double x2 = x * x, term = x * x2, s = 0.0; /* (-1)^{m+1} x^{2m+1}/(m-1)! */
        for (int m = 1; m < 40; ++m) {
            double c = term / (2.0 * m + 1.0);
            s += c;
            if (fabs(c) < 1e-18 * fabs(s))
                break;
            term *= -x2 / m;
        }
        bracket = 4.0 / sqrt(PI) * s / rho;
    } else {
        bracket = erf(x) / rho - exp(-x * x) / sqrt(PI * alpha * delta);
    }
    return (1.0 / (4.0 * PI)) * rn / (rho * rho) * bracket;
}

/* V^d(r): eq. V0 for d = 0, eq. vd for d >= 1. */
double orc_V_d(double rho, int d, double h, double alpha)
{
    if (d == 0)
        return h * orc_G_dtau(rho, 0.0, alpha) - orc_G_dtau_dt(rho, h, alpha) +
               orc_G_dtau_dt(rho, 0.0, alpha);
    return 2.0 * orc_G_dtau_dt(rho, d * h, alpha) -
           orc_G_dtau_dt(rho, (d + 1) * h, alpha) -
           orc_G_dtau_dt(rho, (d - 1) * h, alpha);
}

/* K^d(r): eq. K0 for d = 0, eq. K_d for d >= 1 (scaled forms include alpha). */
double orc_K_d(double rn, double rho, int d, double h, double alpha)
{
    if (d == 0)
        return h * orc_dn_G_dtau(rn, rho, 0.0, alpha) -
               orc_dn_G_dtau_dt(rn, rho, h, alpha) +
               orc_dn_G_dtau_dt(rn, rho, 0.0, alpha);
    return 2.0 * orc_dn_G_dtau_dt(rn, rho, d * h, alpha) -
           orc_dn_G_dtau_dt(rn, rho, (d + 1) * h, alpha) -
           orc_dn_G_dtau_dt(rn, rho, (d - 1) * h, alpha);
}
