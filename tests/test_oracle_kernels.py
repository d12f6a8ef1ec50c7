"""Pins of the oracle's heat-kernel functions against what the paper and the
mathematics fix (not against a retyped formula):

* the heat kernel integrates to one over R^3 (Sec. 2, fundamental solution);
* the scaled normal derivative is alpha times the spatial derivative of G;
* the antiderivatives of Sec. 3 satisfy d/d delta G^{dtau} = -G and
  d/d delta G^{dtau dt} = G^{dtau} (checked as integrals of the lower one);
* eq. dG / eq. dn_G_dtau are alpha d/dn_y of eq. G_dtau_dt / eq. G_dtau;
* the printed limits (tests/golden/limits.txt);
* eq. vd and eq. V0 (and eq. K_d, eq. K0) equal the time integrals of the
  definition eq. V_d, reduced to int (h - |s|) G(r, d h + s) ds.
"""
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
EPS = np.finfo(np.float64).eps


def gl(f, a, b, n=48, pieces=8, grade=None):
    """Composite Gauss-Legendre (numpy's rule) of a scalar function."""
    x, w = np.polynomial.legendre.leggauss(n)
    if grade is None:
        edges = np.linspace(a, b, pieces + 1)
    else:  # geometric grading towards a
        edges = a + (b - a) * np.concatenate([[0.0], grade ** np.arange(pieces - 1, -1, -1.0)])
    tot = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        m, r = 0.5 * (lo + hi), 0.5 * (hi - lo)
        tot += r * sum(wi * f(m + r * xi) for xi, wi in zip(x, w))
    return tot


ALPHAS = [0.1, 0.5, 1.0, 2.0, 10.0]


@pytest.mark.parametrize("alpha", ALPHAS)
@pytest.mark.parametrize("delta", [1e-3, 0.1, 1.0])
def test_heat_kernel_unit_mass(orc, alpha, delta):
    rmax = 16.0 * math.sqrt(alpha * delta)
    mass = gl(lambda r: 4.0 * math.pi * r * r * orc.heat_kernel(r, delta, alpha), 0.0, rmax,
              n=64, pieces=4)
    assert abs(mass - 1.0) < 1e-13


def test_heat_kernel_causal(orc):
    assert orc.heat_kernel(0.3, 0.0, 1.0) == 0.0
    assert orc.heat_kernel(0.3, -1.0, 1.0) == 0.0
    assert orc.dn_heat_kernel(0.1, 0.3, -1.0, 1.0) == 0.0


def _fd(fun, e):
    """4th-order central difference at 0."""
    return (-fun(2 * e) + 8 * fun(e) - 8 * fun(-e) + fun(-2 * e)) / (12 * e)


R_VEC = np.array([0.3, -0.2, 0.5])
N_VEC = np.array([0.6, 0.0, 0.8])


@pytest.mark.parametrize("alpha", [0.5, 2.0])
@pytest.mark.parametrize("delta", [0.05, 0.7])
def test_dn_heat_kernel_is_alpha_normal_derivative(orc, alpha, delta):
    rho = np.linalg.norm(R_VEC)
    # y moves along n_y: r(eps) = r - eps n
    fd = _fd(lambda e: orc.heat_kernel(np.linalg.norm(R_VEC - e * N_VEC), delta, alpha), 1e-3 * rho)
    ref = alpha * fd
    got = orc.dn_heat_kernel(float(R_VEC @ N_VEC), rho, delta, alpha)
    assert abs(got - ref) <= 1e-8 * abs(ref)


RHOS = [1e-3, 0.02, 0.3, 1.1]


@pytest.mark.parametrize("alpha", [0.5, 1.0, 2.0])
@pytest.mark.parametrize("rho", RHOS)
def test_G_dtau_is_time_integral_of_G(orc, alpha, rho):
    # G^{dtau}(r, d1) - G^{dtau}(r, d2) = int_{d1}^{d2} G(r, s) ds
    for d1, d2 in [(1e-3, 0.01), (0.01, 0.3), (0.3, 2.0)]:
        lhs = orc.G_dtau(rho, d1, alpha) - orc.G_dtau(rho, d2, alpha)
        rhs = gl(lambda s: orc.heat_kernel(rho, s, alpha), d1, d2, pieces=48, grade=0.5)
        assert abs(lhs - rhs) <= 1e-12 * abs(rhs) + 1e-15 * abs(orc.G_dtau(rho, d1, alpha))


@pytest.mark.parametrize("alpha", [0.5, 1.0, 2.0])
@pytest.mark.parametrize("rho", RHOS)
def test_G_dtau_dt_is_time_integral_of_G_dtau(orc, alpha, rho):
    # G^{dtau dt}(r, d2) - G^{dtau dt}(r, d1) = int_{d1}^{d2} G^{dtau}(r, s) ds,
    # including d1 = 0 where the printed delta -> 0 limit anchors the constant.
    for d1, d2 in [(0.0, 1e-3), (0.0, 0.05), (0.01, 0.3), (0.3, 2.0)]:
        lhs = orc.G_dtau_dt(rho, d2, alpha) - orc.G_dtau_dt(rho, d1, alpha)
        rhs = gl(lambda s: orc.G_dtau(rho, s, alpha), d1, d2, pieces=48, grade=0.5)
        scale = abs(orc.G_dtau_dt(rho, d2, alpha)) + abs(orc.G_dtau_dt(rho, d1, alpha))
        assert abs(lhs - rhs) <= 1e-12 * abs(rhs) + 4 * EPS * scale


# (rho, delta) pairs spanning x = rho / (2 sqrt(alpha delta)) from 1e-3 to ~20,
# so both the series branch (x < 0.5) and the printed branch are exercised.
X_CASES = [(1e-3, 0.25), (0.02, 0.5), (0.1, 0.05), (0.3, 0.1), (0.6, 0.02), (1.1, 0.003)]


@pytest.mark.parametrize("alpha", [0.5, 1.0, 2.0])
@pytest.mark.parametrize("rho,delta", X_CASES)
def test_dn_G_dtau_dt_is_normal_derivative(orc, alpha, rho, delta):
    r = R_VEC / np.linalg.norm(R_VEC) * rho
    step = 1e-3 * rho
    fd = _fd(lambda e: orc.G_dtau_dt(np.linalg.norm(r - e * N_VEC), delta, alpha), step)
    ref = alpha * fd
    got = orc.dn_G_dtau_dt(float(r @ N_VEC), rho, delta, alpha)
    fd_noise = 4 * EPS * alpha * abs(orc.G_dtau_dt(rho, delta, alpha)) / step
    assert abs(got - ref) <= 1e-8 * abs(ref) + fd_noise


@pytest.mark.parametrize("alpha", [0.5, 2.0])
@pytest.mark.parametrize("rho", [0.05, 0.4])
def test_dn_G_dtau_is_normal_derivative_and_time_integral(orc, alpha, rho):
    r = R_VEC / np.linalg.norm(R_VEC) * rho
    rn = float(r @ N_VEC)
    for delta in [1e-3, 0.05, 0.6]:
        fd = _fd(lambda e: orc.G_dtau(np.linalg.norm(r - e * N_VEC), delta, alpha), 1e-3 * rho)
        ref = alpha * fd
        assert abs(orc.dn_G_dtau(rn, rho, delta, alpha) - ref) <= 1e-8 * abs(ref)
    # alpha dG^{dtau}/dn (d1) - alpha dG^{dtau}/dn (d2) = int alpha dG/dn
    for d1, d2 in [(1e-3, 0.05), (0.05, 1.0)]:
        lhs = orc.dn_G_dtau(rn, rho, d1, alpha) - orc.dn_G_dtau(rn, rho, d2, alpha)
        rhs = gl(lambda s: orc.dn_heat_kernel(rn, rho, s, alpha), d1, d2, pieces=16, grade=0.5)
        assert abs(lhs - rhs) <= 1e-11 * abs(rhs)
    # alpha dG^{dtau dt}/dn (d2) - (d1) = int alpha dG^{dtau}/dn, from d1 = 0 (limit)
    for d1, d2 in [(0.0, 0.02), (0.02, 0.8)]:
        lhs = orc.dn_G_dtau_dt(rn, rho, d2, alpha) - orc.dn_G_dtau_dt(rn, rho, d1, alpha)
        rhs = gl(lambda s: orc.dn_G_dtau(rn, rho, s, alpha), d1, d2, pieces=16, grade=0.5)
        assert abs(lhs - rhs) <= 1e-11 * abs(rhs)


def test_psi_series_matches_printed_form_where_both_are_accurate(orc):
    for x in np.linspace(0.3, 1.5, 25):
        a, b = orc.psi_series(x), orc.psi_direct(x)
        assert abs(a - b) <= 2e-14 * abs(b)


def test_psi_series_high_precision(orc):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    for x in [1e-6, 1e-4, 1e-2, 0.1, 0.3, 0.49]:
        X = mp.mpf(x)
        ref = mp.erf(X) / 2 - mp.erf(X) / (4 * X * X) + mp.exp(-X * X) / (2 * mp.sqrt(mp.pi) * X)
        assert abs(orc.psi_series(x) - float(ref)) <= 4 * EPS * abs(float(ref))


def _load_limits():
    rows = []
    with open(os.path.join(HERE, "golden", "limits.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                p = line.split()
                rows.append((p[0], p[1]) + tuple(float(v) for v in p[2:]))
    return rows


@pytest.mark.parametrize("row", _load_limits(), ids=lambda r: r[0] + "_" + r[1])
def test_printed_limits(orc, row):
    name, which, c, a, b, e, f, p = row
    fun = {"G_dtau_dt": lambda rn, rho, d, al: orc.G_dtau_dt(rho, d, al),
           "G_dtau": lambda rn, rho, d, al: orc.G_dtau(rho, d, al),
           "dn_G_dtau_dt": orc.dn_G_dtau_dt,
           "dn_G_dtau": orc.dn_G_dtau}[name]
    for alpha in [0.5, 1.0, 3.0]:
        for rho, rn in [(0.2, 0.07), (0.9, -0.4)]:
            d_fixed = 0.3
            if which == "delta->0":
                expect = c * rn ** a * rho ** b * alpha ** e * math.pi ** p
                # exactly at delta = 0, and as the limit of the delta > 0 branch:
                # for x >= 42 the exponential terms underflow the result and what
                # remains is affine in delta, so 2 f(d) - f(2 d) is the limit.
                assert fun(rn, rho, 0.0, alpha) == pytest.approx(expect, rel=1e-15, abs=0)
                d_small = (rho / 120.0) ** 2 / alpha
                lim = 2 * fun(rn, rho, d_small, alpha) - fun(rn, rho, 2 * d_small, alpha)
                assert lim == pytest.approx(expect, rel=1e-13, abs=0)
            else:
                expect = c * rn ** a * alpha ** e * d_fixed ** f * math.pi ** p
                assert fun(rn, 0.0, d_fixed, alpha) == pytest.approx(expect, rel=1e-15, abs=0)
                # approach along a ray (rn proportional to rho): the deviation
                # from the limit is small and shrinks at least linearly in rho
                tiny = 1e-5 * math.sqrt(alpha * d_fixed)
                dev1 = abs(fun(rn * tiny, tiny, d_fixed, alpha) - expect)
                dev2 = abs(fun(rn * tiny / 10, tiny / 10, d_fixed, alpha) - expect)
                assert dev1 <= 1e-6 * (abs(expect) + 1.0)
                assert dev2 <= 0.2 * dev1 + 4 * EPS * (abs(expect) + 1.0)


@pytest.mark.parametrize("alpha", [0.5, 1.0, 2.0])
@pytest.mark.parametrize("rho", [0.01, 0.15, 0.6])
def test_second_difference_equals_time_integral(orc, alpha, rho):
    """eq. vd / eq. V0 against int (h-|s|) G(r, dh + s) ds, the reduction of the
    definition eq. V_d; same for eq. K_d / eq. K0 with alpha dG/dn_y.  The
    tolerance is the rounding bound of the printed second difference."""
    h = 1.0 / 16
    r = R_VEC / np.linalg.norm(R_VEC) * rho
    rn = float(r @ N_VEC)
    for d in [0, 1, 2, 5, 15]:
        if d == 0:
            vref = gl(lambda s: (h - s) * orc.heat_kernel(rho, s, alpha), 0.0, h, pieces=24, grade=0.6)
            kref = gl(lambda s: (h - s) * orc.dn_heat_kernel(rn, rho, s, alpha), 0.0, h,
                      pieces=24, grade=0.6)
            vscale = h * orc.G_dtau(rho, 0, alpha) + orc.G_dtau_dt(rho, h, alpha)
            kscale = abs(h * orc.dn_G_dtau(rn, rho, 0, alpha)) + abs(orc.dn_G_dtau_dt(rn, rho, h, alpha))
        else:
            lo = (d - 1) * h
            if d == 1:
                left = gl(lambda s: s * orc.heat_kernel(rho, s, alpha), 0.0, h, pieces=24, grade=0.6)
                kleft = gl(lambda s: s * orc.dn_heat_kernel(rn, rho, s, alpha), 0.0, h,
                           pieces=24, grade=0.6)
            else:
                left = gl(lambda s: (s - lo) * orc.heat_kernel(rho, s, alpha), lo, lo + h, pieces=4)
                kleft = gl(lambda s: (s - lo) * orc.dn_heat_kernel(rn, rho, s, alpha), lo, lo + h,
                           pieces=4)
            right = gl(lambda s: (lo + 2 * h - s) * orc.heat_kernel(rho, s, alpha), lo + h, lo + 2 * h,
                       pieces=4)
            kright = gl(lambda s: (lo + 2 * h - s) * orc.dn_heat_kernel(rn, rho, s, alpha), lo + h,
                        lo + 2 * h, pieces=4)
            vref, kref = left + right, kleft + kright
            vscale = sum(abs(orc.G_dtau_dt(rho, (d + k) * h, alpha)) * (2 if k == 0 else 1)
                         for k in (-1, 0, 1))
            kscale = sum(abs(orc.dn_G_dtau_dt(rn, rho, (d + k) * h, alpha)) * (2 if k == 0 else 1)
                         for k in (-1, 0, 1))
        v = orc.V_d(rho, d, h, alpha)
        k = orc.K_d(rn, rho, d, h, alpha)
        assert abs(v - vref) <= 1e-12 * abs(vref) + 16 * EPS * vscale, (d, v, vref)
        assert abs(k - kref) <= 1e-11 * abs(kref) + 16 * EPS * kscale + 1e-300, (d, k, kref)
