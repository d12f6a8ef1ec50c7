"""Pins of the oracle's piecewise-linear trial space (Sec. 3.2: K_h with the
nodal hat functions phi_i of X_h^{1,0}; Sec. 3.4: the L2(Sigma_h) projection
of the Dirichlet datum into X_h^{1,0} and the right-hand side
(1/2 M_h + K_h) g with the p0 x p1 mass matrix):

* partition of unity: sum_i K1^d[l,i] equals the row sum of the p0 block K^d;
* coplanar zeros: a node whose triangles all lie in the plane of gamma_l
  gets K1^d[l,i] = 0 (r . n_y = 0);
* divergence theorem with a linear density f(y) = c0 + c.y on the cube
  [0,1]^3 (independent closed forms): with P_f(x,s) = int_Omega f G dy and
  grad P(x,s) = int_Omega grad_y G dy,
      int_Gamma alpha dG/dn_y f ds_y = alpha c . grad P + d/ds P_f,
  integrated against the time weight w_d(s) of block d (the hat
  h - |s - dh| for d >= 1, h - s on [0, h] for d = 0), so that
      sum_i K1^d[l,i] f(x_i) = int_{gamma_l} ( int w_d d/ds P_f ds + alpha int w_d c.grad P ds );
  the nodal values f(x_i) interpolate f exactly, so this checks the
  barycentric weights and their node mapping on every pair class;
* the projection is L2-orthogonal: int int (g - g1_h) phi_i = 0 for every
  node, with the moments of g computed here by an independent rule;
* the paper's printed errors of the computed Neumann datum for its two
  coarsest Dirichlet runs (Table dirconv: 8 steps / 192 triangles and
  16 steps / 768 triangles), which used piecewise-linear Dirichlet data
  (tests/golden/table_dirconv.txt).
"""
import math

import numpy as np
import pytest
from scipy.special import erf

import workloads


@pytest.fixture(scope="module")
def cube2p1(orc):
    nodes, tris = workloads.cube_mesh(2)
    alpha, T, n_steps = 1.0, 0.6, 6
    E = len(tris)
    V, K = orc.assemble_rows(nodes, tris, alpha, T, n_steps, np.arange(E))
    K1 = orc.assemble_k1_rows(nodes, tris, alpha, T, n_steps, np.arange(E))
    area, normal = orc.triangle_geometry(nodes, tris)
    return dict(nodes=nodes, tris=tris, alpha=alpha, T=T, n_steps=n_steps, K=K, K1=K1, area=area,
                normal=normal)


def test_partition_of_unity(cube2p1):
    K, K1 = cube2p1["K"], cube2p1["K1"]
    assert np.allclose(K1.sum(axis=2), K.sum(axis=2), rtol=1e-13, atol=1e-15 * np.abs(K).max())


def test_coplanar_nodes_are_zero(cube2p1):
    nodes, tris, normal, K1 = (cube2p1["nodes"], cube2p1["tris"], cube2p1["normal"],
                               cube2p1["K1"])
    hits = 0
    for l in range(len(tris)):
        n_l, p_l = normal[l], nodes[tris[l][0]]
        for i in range(len(nodes)):
            star = [j for j in range(len(tris)) if i in tris[j]]
            coplanar = all(abs(np.dot(nodes[tris[j]] - p_l, n_l)).max() < 1e-14 for j in star)
            if coplanar:
                assert np.all(K1[l, :, i] == 0.0), (l, i)
                hits += 1
    assert hits > 0


def _g1(z, s, alpha):
    return np.exp(-z * z / (4.0 * alpha * s)) / np.sqrt(4.0 * np.pi * alpha * s)


def _P1(x, s, alpha):
    c = np.sqrt(4.0 * alpha * s)
    return 0.5 * (erf((1.0 - x) / c) + erf(x / c))


def _M1(x, s, alpha):  # int_0^1 y g1(x - y) dy
    return x * _P1(x, s, alpha) + 2.0 * alpha * s * (_g1(x, s, alpha) - _g1(x - 1.0, s, alpha))


C0, CV = 2.0, np.array([0.3, -0.5, 0.8])


def _Pf(x, s, alpha):
    """x [..., 3], s broadcast: int_Omega (C0 + CV.y) G(x - y, s) dy."""
    P = [_P1(x[..., i], s, alpha) for i in range(3)]
    M = [_M1(x[..., i], s, alpha) for i in range(3)]
    out = C0 * P[0] * P[1] * P[2]
    for i in range(3):
        others = [P[k] for k in range(3) if k != i]
        out = out + CV[i] * M[i] * others[0] * others[1]
    return out


def _cgradP(x, s, alpha):
    """CV . int_Omega grad_y G(x - y, s) dy."""
    P = [_P1(x[..., i], s, alpha) for i in range(3)]
    out = 0.0
    for i in range(3):
        others = [P[k] for k in range(3) if k != i]
        dG = _g1(x[..., i] - 1.0, s, alpha) - _g1(x[..., i], s, alpha)
        out = out + CV[i] * dG * others[0] * others[1]
    return out


def test_linear_density_divergence_theorem(orc, cube2p1):
    nodes, tris, alpha = cube2p1["nodes"], cube2p1["tris"], cube2p1["alpha"]
    n_steps, h = cube2p1["n_steps"], cube2p1["T"] / cube2p1["n_steps"]
    K1, area = cube2p1["K1"], cube2p1["area"]
    fnode = C0 + nodes @ CV
    S1, S2, W = orc.triangle_rule(10)
    ug, uw = np.polynomial.legendre.leggauss(24)
    ug, uw = 0.5 * (ug + 1.0), 0.5 * uw
    worst = np.zeros(n_steps)
    for l in range(len(tris)):
        P = nodes[tris[l]]
        x = P[0] + S1[:, None] * (P[1] - P[0]) + S2[:, None] * (P[2] - P[1])  # [nq, 3]
        fx = C0 + x @ CV
        for d in range(n_steps):
            # time part: int w_d dP_f/ds ds (graded towards t = 0 for d = 0)
            if d == 0:
                edges = h * np.concatenate([[0.0], 0.25 ** np.arange(11, -1, -1.0)])
                tot = np.zeros(len(x))
                for a, b in zip(edges[:-1], edges[1:]):
                    t = a + (b - a) * ug
                    tot += (b - a) * ((_Pf(x[:, None, :], t[None, :], alpha) - 0.5 * fx[:, None])
                                      @ uw)
            else:
                t = (d + ug) * h
                tot = h * ((_Pf(x[:, None, :], t[None, :], alpha) -
                            _Pf(x[:, None, :], (t - h)[None, :], alpha)) @ uw)
            # gradient part: alpha int w_d(s) c.gradP(x, s) ds, s = u^2 near 0
            lo, hi = max(0.0, (d - 1) * h), (d + 1) * h if d > 0 else h
            grad = np.zeros(len(x))
            pieces = [(lo, d * h), (d * h, hi)] if d > 0 else [(0.0, h)]
            for a, b in pieces:
                if b <= a:
                    continue
                ua, ub = math.sqrt(a), math.sqrt(b)
                u = ua + (ub - ua) * ug
                s = u * u
                wd = h - np.abs(s - d * h) if d > 0 else h - s
                grad += (ub - ua) * ((_cgradP(x[:, None, :], s[None, :], alpha) * (2.0 * u * wd))
                                     @ uw)
            exact = 2.0 * area[l] * np.dot(W, tot + alpha * grad)
            got = np.dot(K1[l, d], fnode)
            worst[d] = max(worst[d], abs(got - exact) / max(abs(exact), 1e-300))
    # quadrature error of the q = 3 / m = 4 rules, as for the constant density
    # (observed there: 6e-4 at d = 0 falling to 7e-7); a wrong weight or node
    # mapping is an O(1) deviation
    assert np.all(worst < np.array([3e-3, 3e-4, 5e-5, 2e-5, 1e-5, 5e-6])), worst


def test_projection_is_l2_orthogonal(orc):
    nodes, tris = workloads.cube_mesh(2)
    alpha, T, n_steps = 0.8, 0.5, 3
    src = workloads.point_source((1.4, 0.3, 0.6), t0=-0.05)
    g1 = orc.project_dirichlet_p1(nodes, tris, alpha, T, n_steps, src)[0]
    area, _ = orc.triangle_geometry(nodes, tris)
    S1, S2, W = orc.triangle_rule(12)
    tg, tw = np.polynomial.legendre.leggauss(20)
    tg, tw = 0.5 * (tg + 1.0), 0.5 * tw
    h = T / n_steps
    y, t0 = np.array([1.4, 0.3, 0.6]), -0.05
    N = len(nodes)
    for k in range(n_steps):
        b = np.zeros(N)
        mass = np.zeros(N)
        for j, t3 in enumerate(tris):
            P = nodes[t3]
            x = P[0] + S1[:, None] * (P[1] - P[0]) + S2[:, None] * (P[2] - P[1])
            lam = np.stack([1.0 - S1, S1 - S2, S2], axis=1)
            t = (k + tg) * h - t0
            r2 = ((x - y) ** 2).sum(axis=1)
            G = np.exp(-r2[:, None] / (4 * alpha * t[None, :])) / (4 * np.pi * alpha * t[None, :]) ** 1.5
            gbar = G @ tw  # time mean over the step
            gh = lam @ g1[k][t3]  # the projection at the points
            for v in range(3):
                b[t3[v]] += 2.0 * area[j] * np.dot(W, gbar * lam[:, v])
                mass[t3[v]] += 2.0 * area[j] * np.dot(W, gh * lam[:, v])
        assert np.abs(mass - b).max() <= 1e-9 * np.abs(b).max(), k


@pytest.mark.parametrize("row", [0, 1])
def test_table_dirconv_computed_with_p1_data(orc, row):
    """The two coarsest rows of Table dirconv (cube (-1,1)^3, 192 / 768
    triangles, 8 / 16 steps, alpha = 0.5, source (0,0,1.5)) with the paper's
    own discretisation of the data: the computed error must match the printed
    6.07e-1 / 4.28e-1 within 2 % (the quadrature orders and the diagonal
    direction of the squares are not printed; the p0-data variant gives
    0.599 / 0.423).  Rows of the blocks are assembled on host threads."""
    from concurrent.futures import ThreadPoolExecutor

    import test_oracle_solve
    n_steps, E, comp, proj = test_oracle_solve.load_dirconv()[row]
    alpha, T = 0.5, 1.0
    src = workloads.point_source((0.0, 0.0, 1.5), t0=0.0)
    nodes, tris = workloads.cube_mesh(int(round(math.sqrt(E / 12))), lo=-1.0, hi=1.0)
    assert len(tris) == E
    chunks = np.array_split(np.arange(E), 8)
    with ThreadPoolExecutor(8) as ex:
        V = list(ex.map(lambda r: orc.assemble_rows(nodes, tris, alpha, T, n_steps, r)[0], chunks))
        K1 = list(ex.map(lambda r: orc.assemble_k1_rows(nodes, tris, alpha, T, n_steps, r), chunks))
    V = np.ascontiguousarray(np.concatenate(V).transpose(1, 0, 2))
    K1 = np.ascontiguousarray(np.concatenate(K1).transpose(1, 0, 2))
    area, _ = orc.triangle_geometry(nodes, tris)
    g1 = orc.project_dirichlet_p1(nodes, tris, alpha, T, n_steps, src)
    w = orc.dirichlet_solve(V, orc.dirichlet_rhs_p1(area, tris, K1, g1, T))
    e2, r2 = orc.neumann_error(nodes, tris, alpha, T, n_steps, src, w)
    err = math.sqrt(e2 / r2)
    assert abs(err - comp) < 0.02 * comp, err
