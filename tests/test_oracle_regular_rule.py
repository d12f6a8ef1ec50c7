"""The oracle's regular rule on separated pairs (Sec. 3.1, eq. quad_reg and the
triangle rule of eq. st) against brute-force composite quadrature.

For a disjoint pair the spatial sums S_i = int_{gamma_l} int_{gamma_j} k(x - y)
of the time-level antiderivatives (eq. G_dtau_dt and its normal derivative
eq. dG, at delta = i h, and the delta = 0 terms 1/(4 pi alpha rho) and
r.n_y/(4 pi rho^3)) have smooth integrands.  The reference here shares
nothing with the oracle's rule: each triangle is cut into 4^L congruent
pieces by midpoint subdivision and every piece gets a Gauss-Legendre rule
collapsed onto the triangle along the other edge (numpy's nodes), with the
kernels evaluated in numpy and checked pointwise against the oracle's
scalar kernels.  The oracle's conical rule of order q must converge to it
monotonically and reach it to rounding for the pairs that are well apart.
"""
import numpy as np
import pytest
from scipy.special import erf

import oracle
import workloads

ALPHA, H, N_LEV = 1.0, 0.05, 4


def k_v(rho, delta):
    """G^{d tau d t}(rho, delta) (eq. G_dtau_dt; rho / (8 pi alpha^2) at delta = 0)."""
    if delta == 0.0:
        return rho / (8 * np.pi * ALPHA ** 2)
    x = rho / (2 * np.sqrt(ALPHA * delta))
    return (np.sqrt(delta) / (4 * np.pi * ALPHA ** 1.5) *
            ((x + 0.5 / x) * erf(x) + np.exp(-x * x) / np.sqrt(np.pi)))


def k_k(rn, rho, delta):
    """alpha dG^{d tau d t}/dn_y with rn = (x - y).n_y: -rn/(8 pi alpha rho) phi'(x)."""
    if delta == 0.0:
        return -rn / (8 * np.pi * ALPHA * rho)
    x = rho / (2 * np.sqrt(ALPHA * delta))
    return (-rn / (8 * np.pi * ALPHA * rho) *
            ((1 - 0.5 / x ** 2) * erf(x) + np.exp(-x * x) / (np.sqrt(np.pi) * x)))


def composite_points(v, L, n):
    """Points and weights of the composite rule on the triangle v (3 x 3)."""
    u, wu = np.polynomial.legendre.leggauss(n)
    u, wu = (u + 1) / 2, wu / 2
    pieces = [tuple(v)]
    for _ in range(L):
        nxt = []
        for a, b, c in pieces:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        pieces = nxt
    X, W = [], []
    xi, t = np.repeat(u, n), np.tile(u, n)
    wq = np.repeat(wu, n) * np.tile(wu, n) * (1 - xi)
    for a, b, c in pieces:
        two_area = np.linalg.norm(np.cross(b - a, c - a))
        X.append(a + np.outer(xi, b - a) + np.outer((1 - xi) * t, c - a))
        W.append(wq * two_area)
    return np.vstack(X), np.concatenate(W)


def reference_sums(vl, vj, nj, L, n):
    X, WX = composite_points(vl, L, n)
    Y, WY = composite_points(vj, L, n)
    r = X[:, None, :] - Y[None, :, :]
    rho = np.linalg.norm(r, axis=2)
    rn = r @ nj
    W = WX[:, None] * WY[None, :]
    SV = [np.sum(W * k_v(rho, i * H)) for i in range(N_LEV)]
    SK = [np.sum(W * k_k(rn, rho, i * H)) for i in range(N_LEV)]
    SV.append(np.sum(W / (4 * np.pi * ALPHA * rho)))
    SK.append(np.sum(W * rn / (4 * np.pi * rho ** 3)))
    return np.array(SV), np.array(SK)


def test_numpy_kernels_match_the_oracle(orc):
    for rn, rho, d in ((0.3, 0.5, 0.05), (-0.2, 0.9, 0.2), (0.1, 0.4, 0.0), (0.0, 2.0, 0.15)):
        assert np.isclose(k_v(rho, d), orc.G_dtau_dt(rho, d, ALPHA), rtol=1e-14, atol=0)
        assert np.isclose(k_k(rn, rho, d), orc.dn_G_dtau_dt(rn, rho, d, ALPHA), rtol=1e-14,
                          atol=1e-300)
        assert np.isclose(rn / (4 * np.pi * rho ** 3), orc.dn_G_dtau(rn, rho, 0.0, ALPHA),
                          rtol=1e-14, atol=1e-300)


def _pairs():
    """The closest, a middle and the farthest disjoint pair of the 48-triangle cube."""
    nodes, tris = workloads.cube_mesh(2)
    cent = nodes[tris].mean(axis=1)
    E = len(tris)
    cand = []
    for l in range(E):
        for j in range(E):
            if l != j and oracle.pair_class(tris[l], tris[j])[0] == 0:
                cand.append((float(np.linalg.norm(cent[l] - cent[j])), l, j))
    cand.sort()
    return nodes, tris, [cand[0], cand[len(cand) // 2], cand[-1]]


@pytest.mark.parametrize("which", [0, 1, 2])
def test_regular_rule_converges_to_composite_reference(orc, which):
    nodes, tris, pairs = _pairs()
    dist, l, j = pairs[which]
    _, normal = orc.triangle_geometry(nodes, tris)
    vl, vj = nodes[tris[l]], nodes[tris[j]]
    RV, RK = reference_sums(vl, vj, normal[j], 2, 10)
    CV, CK = reference_sums(vl, vj, normal[j], 1, 14)  # the reference against itself
    assert np.abs(CV - RV).max() <= 1e-14 * np.abs(RV).max()
    assert np.abs(CK - RK).max() <= 1e-14 * max(np.abs(RK).max(), 1e-300) + 1e-300
    coplanar = abs(abs(np.dot(normal[l], normal[j])) - 1.0) < 1e-12 and \
        abs(np.dot(vl[0] - vj[0], normal[j])) < 1e-12
    if coplanar:
        assert np.abs(RK).max() <= 1e-15 * np.abs(RV).max()
    errs = []
    for q in range(2, 10):
        SV, SK = orc.pair_sums(nodes, tris, l, j, ALPHA, H, N_LEV, q_reg=q)
        e = (np.abs(SV - RV) / np.abs(RV)).max()
        if not coplanar:
            e = max(e, (np.abs(SK - RK) / np.abs(RK)).max())
        else:
            assert np.abs(SK).max() <= 1e-15 * np.abs(SV).max()
        errs.append(e)
    errs = np.array(errs)
    print("pair (%d, %d), centroid distance %.3f: rel. error q=2..9 %s"
          % (l, j, dist, " ".join("%.1e" % e for e in errs)))
    # monotone down to the rounding floor
    for a, b in zip(errs[:-1], errs[1:]):
        assert b <= a or b <= 1e-13, errs
    assert errs[0] > 1e3 * max(errs[-1], 1e-15)  # it really converges (not a copy of the reference)
    if which == 0:  # the closest pair (adjacent faces, nearly touching): algebraic rate
        assert errs[6] <= 2e-8 and errs[7] <= 2e-9, errs
    else:
        assert errs[6] <= 1e-12, errs
