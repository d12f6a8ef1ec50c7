"""Pins of the oracle's assembly of V^d and K^d (Sec. 3.1-3.2, Sec. 5):

* V^d is symmetric to rounding (radial kernel, same p0 space for test and
  trial; a touching pair's regularised rule serves both entries); V^0 is
  positive definite;
* K^d vanishes on coplanar pairs (r . n_y = 0 on a flat face);
* the blocks depend on h and d only: a run with half the steps and half the
  horizon reproduces the leading blocks bit for bit;
* the blocks are the combinations of the time-level sums given by Table deltad
  and eq. vd / eq. V0 (tests/golden/table_deltad.txt), recovered by least
  squares from the oracle's own sums;
* divergence theorem on the cube [0,1]^3 (row sums of K): with
  P(x,s) = int_Omega G(x-y,s) dy = prod_i (erf((1-x_i)/sqrt(4 alpha s)) + erf(x_i/sqrt(4 alpha s)))/2
  and d/ds G = alpha Lap G,  int_Gamma alpha dG/dn_y(x-y,s) ds_y = dP/ds, so
     sum_j K^d[l,j] = int_{gamma_l} int_{dh}^{(d+1)h} P(x,t) - P(x,t-h) dt   (d >= 1)
     sum_j K^0[l,j] = int_{gamma_l} int_0^h P(x,t) - 1/2 dt                  (x in a face).
"""
import math
import os

import numpy as np
import pytest
from scipy.special import erf

import workloads

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def cube2(orc):
    nodes, tris = workloads.cube_mesh(2)
    alpha, T, n_steps = 1.0, 0.6, 6
    V, K, SV, SK = orc.assemble_rows(nodes, tris, alpha, T, n_steps, np.arange(len(tris)),
                                     with_sums=True)
    area, normal = orc.triangle_geometry(nodes, tris)
    return dict(nodes=nodes, tris=tris, alpha=alpha, T=T, n_steps=n_steps, V=V, K=K,
                SV=SV, SK=SK, area=area, normal=normal)


def touching_mask(tris):
    E = len(tris)
    m = np.zeros((E, E), dtype=bool)
    for a in range(E):
        for b in range(E):
            m[a, b] = len(set(tris[a]) & set(tris[b])) > 0
    return m


EPS = np.finfo(np.float64).eps


def cond_scale(S, d, h):
    """Magnitude of the terms of the second difference giving block d:
    |S_{d-1}| + 2|S_d| + |S_{d+1}| (d >= 1), h|S_*| + |S_1| + |S_0| (d = 0)."""
    A = np.abs(S)
    if d == 0:
        return h * A[:, -1, :] + A[:, 1, :] + A[:, 0, :]
    return A[:, d - 1, :] + 2 * A[:, d, :] + A[:, d + 1, :]


def test_V_symmetric(cube2):
    V = cube2["V"].transpose(1, 0, 2)  # [d][l][j]
    h = cube2["T"] / cube2["n_steps"]
    for d in range(V.shape[0]):
        A = V[d]
        asym = np.abs(A - A.T)
        c = cond_scale(cube2["SV"], d, h)
        rounding = 8 * EPS * np.maximum(c, c.T)
        assert np.all(asym <= rounding), d


def test_V0_positive_definite(cube2):
    V0 = cube2["V"][:, 0, :]
    ev = np.linalg.eigvalsh(0.5 * (V0 + V0.T))
    assert ev.min() > 0


def test_K_vanishes_on_coplanar_pairs(cube2):
    K = cube2["K"].transpose(1, 0, 2)
    n = cube2["normal"]
    coplanar = np.abs(n @ n.T - 1.0) < 1e-12
    # same face of the cube: same normal and the same plane offset
    nodes, tris = cube2["nodes"], cube2["tris"]
    off = np.einsum("ij,ij->i", n, nodes[tris[:, 0]])
    coplanar &= np.abs(off[:, None] - off[None, :]) < 1e-12
    scale = np.abs(K).max()
    assert np.abs(K[:, coplanar]).max() <= 1e-13 * scale
    assert np.abs(K[:, ~coplanar]).max() > 1e-3 * scale


def test_toeplitz_prefix_is_independent_of_horizon(orc, cube2):
    nodes, tris = cube2["nodes"], cube2["tris"]
    rows = np.array([0, 5, 17, 40])
    V2, K2 = orc.assemble_rows(nodes, tris, cube2["alpha"], cube2["T"] / 2, cube2["n_steps"] // 2,
                               rows)
    assert np.array_equal(V2, cube2["V"][rows, : cube2["n_steps"] // 2])
    assert np.array_equal(K2, cube2["K"][rows, : cube2["n_steps"] // 2])


def load_deltad():
    table = {}
    with open(os.path.join(HERE, "golden", "table_deltad.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            it, rest = line.split(":", 1)
            table[int(it)] = {int(a): float(b) for a, b in (p.split(":") for p in rest.split())}
    return table


def test_blocks_follow_table_deltad(cube2):
    table = load_deltad()
    n_steps = cube2["n_steps"]
    assert max(table) == n_steps
    h = cube2["T"] / n_steps
    for name, S, A in (("V", cube2["SV"], cube2["V"]), ("K", cube2["SK"], cube2["K"])):
        X = S.transpose(0, 2, 1).reshape(-1, n_steps + 2)  # samples x (levels 0..E_t, singular)
        keep = np.abs(X).sum(1) > 0
        X = X[keep]
        for d in range(n_steps):
            y = A[:, d, :].reshape(-1)[keep]
            coef, *_ = np.linalg.lstsq(X, y, rcond=None)
            expect = np.zeros(n_steps + 2)
            for it, row in table.items():
                if d in row:
                    expect[it] = row[d]
            if d == 0:
                expect[n_steps + 1] = h  # eq. V0 / eq. K0: h times the delta = 0 integral
            assert np.allclose(coef, expect, atol=1e-6), (name, d, coef, expect)


def cube_P(x, s, alpha):
    c = np.sqrt(4.0 * alpha * s)
    return np.prod(0.5 * (erf((1.0 - x) / c) + erf(x / c)), axis=-1)


def test_K_row_sums_divergence_theorem(orc, cube2):
    nodes, tris, alpha = cube2["nodes"], cube2["tris"], cube2["alpha"]
    n_steps, h = cube2["n_steps"], cube2["T"] / cube2["n_steps"]
    S1, S2, W = orc.triangle_rule(10)
    tg, tw = np.polynomial.legendre.leggauss(24)
    tg, tw = 0.5 * (tg + 1.0), 0.5 * tw
    K = cube2["K"]
    worst = np.zeros(n_steps)
    for l in range(len(tris)):
        P = nodes[tris[l]]
        area = cube2["area"][l]
        x = P[0] + S1[:, None] * (P[1] - P[0]) + S2[:, None] * (P[2] - P[1])
        for d in range(n_steps):
            if d == 0:
                # graded in t towards 0 where P(x, t) leaves 1/2 in thin layers
                edges = h * np.concatenate([[0.0], 0.25 ** np.arange(11, -1, -1.0)])
                tot = 0.0
                for a, b in zip(edges[:-1], edges[1:]):
                    t = a + (b - a) * tg
                    vals = cube_P(x[:, None, :], t[None, :, None], alpha) - 0.5
                    tot += (b - a) * np.sum(W[:, None] * tw[None, :] * vals)
            else:
                t = (d + tg) * h
                vals = cube_P(x[:, None, :], t[None, :, None], alpha) - cube_P(
                    x[:, None, :], (t - h)[None, :, None], alpha)
                tot = h * np.sum(W[:, None] * tw[None, :] * vals)
            exact = 2.0 * area * tot
            got = K[l, d, :].sum()
            worst[d] = max(worst[d], abs(got - exact) / max(abs(exact), 1e-300))
    # the discrete sums carry the spatial quadrature error of the q = 3 / m = 4
    # rules; a wrong sign, factor or dropped term is an O(1) deviation
    # (observed: 6e-4 at d = 0 falling to 7e-7 at d = 5; bounds ~5x that)
    assert np.all(worst < np.array([3e-3, 3e-4, 5e-5, 2e-5, 1e-5, 5e-6])), worst
