"""Pins of the oracle's quadrature rules:

* Gauss rules and the conical triangle rule integrate monomials exactly up to
  their degree (closed-form moments);
* the regularised rules for touching pairs (eq. quad_duffy, eq. ss) put every
  point inside T x T, integrate the constant to |T|^2 = 1/4 and low-degree
  polynomials exactly;
* for the singular pair integrals of V^0 and K^0 at delta = 0
  (int int 1/|x-y| and int int (x-y).n_y/|x-y|^3 over touching pairs) the
  oracle's pair sums converge, as the order grows, to references built from
  closed-form inner integrals (the potential of a uniform flat triangle and the
  signed solid angle of a triangle) integrated by a fine composite rule.
"""
import math

import numpy as np
import pytest

EPS = np.finfo(np.float64).eps


@pytest.mark.parametrize("n", range(1, 13))
def test_gauss_legendre_moments(orc, n):
    x, w = orc.gauss_legendre01(n)
    assert np.all(np.diff(x) > 0) and x[0] > 0 and x[-1] < 1 and np.all(w > 0)
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 16 * EPS
    # not exact one degree higher (for n >= 1)
    assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-6 / 10 ** n


@pytest.mark.parametrize("n", range(1, 13))
def test_gauss_jacobi_moments(orc, n):
    x, w = orc.gauss_jacobi01(n)  # weight x on [0, 1]
    assert np.all(np.diff(x) > 0) and x[0] > 0 and x[-1] < 1 and np.all(w > 0)
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 2)) < 16 * EPS


def tri_moment(a, b):
    """int_T s1^a s2^b ds over T = {0 <= s2 <= s1 <= 1}."""
    return 1.0 / ((b + 1) * (a + b + 2))


@pytest.mark.parametrize("q", range(1, 9))
def test_triangle_rule_exactness(orc, q):
    s1, s2, w = orc.triangle_rule(q)
    assert np.all((s2 >= 0) & (s2 <= s1) & (s1 <= 1)) and np.all(w > 0)
    for a in range(2 * q):
        for b in range(2 * q - a):
            assert abs(np.sum(w * s1 ** a * s2 ** b) - tri_moment(a, b)) < 16 * EPS


@pytest.mark.parametrize("cls", [1, 2, 3])
@pytest.mark.parametrize("m", [2, 3, 4, 5])
def test_ss_rule_domain_and_polynomials(orc, cls, m):
    s1, s2, t1, t2, w = orc.ss_rule(cls, m)
    tol = 1e-14
    assert np.all((s2 >= -tol) & (s2 <= s1 + tol) & (s1 <= 1 + tol))
    assert np.all((t2 >= -tol) & (t2 <= t1 + tol) & (t1 <= 1 + tol))
    assert np.all(w > 0)
    assert abs(w.sum() - 0.25) < 64 * EPS
    # the maps are polynomial and the Jacobians have degree 3 in zeta, so a
    # monomial of total degree k is integrated exactly when k + 3 <= 2m - 1
    for a, b, c, d in [(1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 1), (1, 0, 1, 0), (2, 0, 0, 1),
                       (1, 1, 1, 0), (0, 2, 0, 2), (2, 1, 1, 2)]:
        if a + b + c + d > 2 * m - 4:
            continue
        exact = tri_moment(a, b) * tri_moment(c, d)
        got = np.sum(w * s1 ** a * s2 ** b * t1 ** c * t2 ** d)
        assert abs(got - exact) < 1e-13, (a, b, c, d, got, exact)


def test_ss_rule_regions_cover_the_identical_pair(orc):
    """Brute-force check that the six identical-pair cones tile T x T: a smooth
    non-polynomial integrand agrees with a fine product rule."""
    s1, s2, t1, t2, w = orc.ss_rule(3, 8)
    f = lambda a, b, c, d: np.exp(0.3 * a - 0.7 * b + 0.2 * c * d) * np.cos(a - d)
    got = np.sum(w * f(s1, s2, t1, t2))
    S1, S2, W = orc.triangle_rule(12)
    ref = np.sum(W[:, None] * W[None, :] * f(S1[:, None], S2[:, None], S1[None, :], S2[None, :]))
    assert abs(got - ref) < 1e-12


# ---------------------------------------------------------------------------
# closed-form inner integrals over a flat triangle (vectorised over points x)
def tri_frame(P):
    P = np.asarray(P, dtype=np.float64)
    n = np.cross(P[1] - P[0], P[2] - P[0])
    area = 0.5 * np.linalg.norm(n)
    return P, n / np.linalg.norm(n), area


def potential_1_over_r(P, x):
    """int_T 1/|x - y| dS_y for a flat CCW triangle P (edge-wise closed form:
    in-plane distances to the edge lines plus the height above the plane)."""
    P, nh, _ = tri_frame(P)
    x = np.atleast_2d(x)
    d = (x - P[0]) @ nh
    proj = x - d[:, None] * nh
    ad = np.abs(d)
    tot = np.zeros(x.shape[0])
    for i in range(3):
        a, b = P[i], P[(i + 1) % 3]
        s_hat = (b - a) / np.linalg.norm(b - a)
        m_hat = np.cross(s_hat, nh)
        p0 = (a - proj) @ m_hat
        sm, sp = (a - proj) @ s_hat, (b - proj) @ s_hat
        rm, rp = np.linalg.norm(x - a, axis=1), np.linalg.norm(x - b, axis=1)
        r02 = p0 * p0 + d * d
        # log((rp + sp) / (rm + sm)) written without cancellation for sm < 0
        num = np.where(sp > 0, rp + sp, r02 / np.maximum(rp - sp, 1e-300))
        den = np.where(sm > 0, rm + sm, r02 / np.maximum(rm - sm, 1e-300))
        tot += p0 * np.log(num / den)
        tot -= ad * (np.arctan2(p0 * sp, r02 + ad * rp) - np.arctan2(p0 * sm, r02 + ad * rm))
    return tot


def double_layer(P, x):
    """int_T (x - y) . n_y / |x - y|^3 dS_y = minus the signed solid angle of T
    seen from x (Van Oosterom-Strackee)."""
    P, _, _ = tri_frame(P)
    x = np.atleast_2d(x)
    a, b, c = P[0] - x, P[1] - x, P[2] - x
    la, lb, lc = (np.linalg.norm(v, axis=1) for v in (a, b, c))
    num = np.einsum("ij,ij->i", a, np.cross(b, c))
    den = la * lb * lc + np.einsum("ij,ij->i", a, b) * lc + np.einsum("ij,ij->i", a, c) * lb \
        + np.einsum("ij,ij->i", b, c) * la
    return -2.0 * np.arctan2(num, den)


def chi(P, s1, s2):
    P = np.asarray(P)
    return P[0] + s1[:, None] * (P[1] - P[0]) + s2[:, None] * (P[2] - P[1])


def composite_points(P, q, k):
    """Points and weights (summing to the area) of a composite conical rule:
    T split into k^2 congruent sub-triangles."""
    import oracle
    S1, S2, W = oracle.triangle_rule(q)
    P, _, area = tri_frame(P)
    pts, wts = [], []
    for i in range(k):
        for j in range(k):
            # sub-triangles of the reference triangle in barycentric grid
            for up in (0, 1):
                if up == 0 and j > i:
                    continue
                if up == 1 and j >= i:
                    continue
                if up == 0:
                    c = [(i, j), (i + 1, j), (i + 1, j + 1)]
                else:
                    c = [(i, j), (i + 1, j + 1), (i, j + 1)]
                c = np.asarray(c, dtype=float) / k
                # map T -> sub-triangle (affine, same orientation convention)
                sub = c[0] + S1[:, None] * (c[1] - c[0]) + S2[:, None] * (c[2] - c[1])
                pts.append(chi(P, sub[:, 0], sub[:, 1]))
                wts.append(W * 2.0 * area / k ** 2)
    return np.concatenate(pts), np.concatenate(wts)


def test_closed_forms_against_plain_quadrature_far_away():
    P = np.array([[0.0, 0.0, 0.0], [1.0, 0.2, 0.0], [0.3, 0.9, 0.1]])
    x = np.array([[1.4, 2.0, 1.5], [-1.0, 0.5, -2.0]])
    y, w = composite_points(P, 8, 2)
    n = tri_frame(P)[1]
    for xi, pot, dl in zip(x, potential_1_over_r(P, x), double_layer(P, x)):
        r = xi - y
        rho = np.linalg.norm(r, axis=1)
        assert abs(pot - np.sum(w / rho)) < 1e-12 * abs(pot)
        assert abs(dl - np.sum(w * (r @ n) / rho ** 3)) < 1e-10 * abs(dl)


PAIRS = {
    # name: (nodes, tris, l, j)
    "identical": (np.array([[0.0, 0, 0], [1.0, 0.1, 0], [0.2, 0.8, 0]]), np.array([[0, 1, 2]]), 0, 0),
    "edge_coplanar": (np.array([[0.0, 0, 0], [1.0, 0, 0], [0.3, 0.8, 0], [0.6, -0.7, 0]]),
                      np.array([[0, 1, 2], [1, 0, 3]]), 0, 1),
    "edge_90deg": (np.array([[0.0, 0, 0], [1.0, 0, 0], [0.4, 0.9, 0], [0.5, 0, 0.8]]),
                   np.array([[0, 1, 2], [1, 0, 3]]), 0, 1),
    "vertex_bent": (np.array([[0.0, 0, 0], [1.0, 0.2, 0], [0.3, 0.9, 0], [-0.8, 0.1, 0.5],
                              [-0.2, -0.9, 0.4]]),
                    np.array([[0, 1, 2], [0, 3, 4]]), 0, 1),
}


def reference_pair(nodes, tris, l, j, kind):
    Pl, Pj = nodes[tris[l]], nodes[tris[j]]
    x, w = composite_points(Pl, 10, 24)
    inner = potential_1_over_r(Pj, x) if kind == "V" else double_layer(Pj, x)
    return np.sum(w * inner)


@pytest.mark.parametrize("name", list(PAIRS))
def test_singular_pair_integrals_converge_to_reference(orc, name):
    nodes, tris, l, j = PAIRS[name]
    alpha, h = 1.0, 0.1
    refV = reference_pair(nodes, tris, l, j, "V") / (4 * math.pi * alpha)
    errs_v, errs_k = [], []
    for m in (3, 5, 8):
        SV, SK = orc.pair_sums(nodes, tris, l, j, alpha, h, 1, q_reg=3, m_ss=m)
        errs_v.append(abs(SV[1] - refV) / abs(refV))
        if name.startswith("identical") or "coplanar" in name:
            assert SK[1] == 0.0 or abs(SK[1]) < 1e-12 * abs(SV[1])
        else:
            refK = reference_pair(nodes, tris, l, j, "K") / (4 * math.pi)
            errs_k.append(abs(SK[1] - refK) / abs(refK))
    assert errs_v[-1] < 1e-7 and errs_v[-1] < errs_v[0], errs_v
    if errs_k:
        assert errs_k[-1] < 1e-6 and errs_k[-1] < errs_k[0], errs_k


@pytest.mark.parametrize("name", ["edge_90deg", "vertex_bent"])
def test_singular_pair_rho_kernel(orc, name):
    """The delta = 0 integrand rho / (8 pi alpha^2) of V^0 (continuous but not
    smooth at touching points) against the composite reference."""
    nodes, tris, l, j = PAIRS[name]
    Pl, Pj = nodes[tris[l]], nodes[tris[j]]
    x, wx = composite_points(Pl, 6, 12)
    y, wy = composite_points(Pj, 6, 12)
    ref = np.sum(wx[:, None] * wy[None, :] * np.linalg.norm(x[:, None] - y[None], axis=2))
    SV, _ = orc.pair_sums(nodes, tris, l, j, 1.0, 0.1, 1, m_ss=6)
    assert abs(SV[0] * 8 * math.pi - ref) < 2e-7 * ref
