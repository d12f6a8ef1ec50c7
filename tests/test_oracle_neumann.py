"""Pins of the oracle's hypersingular operator D_h = D_h^1 + D_h^2 and of
the Neumann problem D_h u = (1/2 M_h^{T_x} - K_h^{T_x}) h (Sec. 3.3, 3.4):

* every block D^d is symmetric, D^0 is positive definite;
* D^1 annihilates constants (the surface curls of the hat functions of a
  triangle sum to the curl of 1, zero);
* the quadratic form of D^1 for the interpolant of a linear function
  u(y) = c . y, whose surface curl on a flat triangle is n x c: fixed by the
  triangles' normals and V alone, independent of the edge formula of the
  curls;
* row sums of D^2 on the unit cube by the divergence theorem:
      sum_j D^{2,d}[i][j] = - int_Gamma phi_i(x) n_x . grad Q_d(x) ds_x,
  Q_d(x) = int_Omega D^{2,d}(x - y) dy = alpha (int_{dh}^{(d+1)h} P -
  int_{(d-1)h}^{dh} P) (d >= 1), alpha int_0^h P (d = 0), P(x,s) =
  int_Omega G(x-y, s) dy in closed form;
* the Neumann right-hand side against the Dirichlet one by the identity
  <g, K^{T_x} h> = <h, R K R g> (R reverses the steps) and the masses;
* the L2(Sigma_h) error of piecewise-linear data: the projection is
  orthogonal in the rule's inner product, so err^2(g1 + e v) - err^2(g1) =
  e^2 ||v||^2 with the exact hat-function mass;
* Table neuconv (tests/golden/table_neuconv.txt), coarsest run: the
  computed error within 2 %, the projected one within 5 %.  (The
  representation column comes out 2-19 % above the printed values: tests
  on the GPU.)
"""
import math

import numpy as np
import pytest

import workloads
from test_oracle_potentials import _P1, _g1

ALPHA = 0.7


@pytest.fixture(scope="module")
def cube3d(orc):
    nodes, tris = workloads.cube_mesh(3)
    T, n_steps = 0.6, 5
    E = len(tris)
    V, _ = orc.assemble(nodes, tris, ALPHA, T, n_steps)
    D1 = orc.assemble_d1(nodes, tris, ALPHA, V)
    D2 = orc.assemble_d2(nodes, tris, ALPHA, T, n_steps)
    return dict(nodes=nodes, tris=tris, T=T, n_steps=n_steps, V=V, D1=D1, D2=D2, E=E)


def test_blocks_symmetric_and_first_block_spd(cube3d):
    D = cube3d["D1"] + cube3d["D2"]
    for d in range(cube3d["n_steps"]):
        # the second differences of later blocks cancel: rounding ~ eps |G^{dtau}|
        assert np.abs(D[d] - D[d].T).max() <= 1e-11 * np.abs(D[d]).max(), d
    assert np.linalg.eigvalsh(D[0]).min() > 0.0


def test_d1_annihilates_constants(cube3d):
    D1 = cube3d["D1"]
    for d in range(cube3d["n_steps"]):
        assert np.abs(D1[d].sum(axis=1)).max() <= 1e-13 * np.abs(D1[d]).max(), d


def test_d1_quadratic_form_of_a_linear_function(orc, cube3d):
    nodes, tris, V, D1 = cube3d["nodes"], cube3d["tris"], cube3d["V"], cube3d["D1"]
    _, normal = orc.triangle_geometry(nodes, tris)
    c = np.array([0.3, -1.1, 0.6])
    u = nodes @ c
    curl = np.cross(normal, c)  # n x c per triangle
    for d in range(cube3d["n_steps"]):
        ref = ALPHA ** 2 * np.einsum("no,nm,mo->", curl, V[d], curl)
        got = u @ D1[d] @ u
        assert abs(got - ref) <= 1e-12 * np.abs(ALPHA ** 2 * np.einsum("no,nm,mo->", np.abs(curl),
                                                                        np.abs(V[d]), np.abs(curl))), d


def _gradP(x, s):
    """grad_x P(x, s) on the unit cube (x [.., 3], s scalar)."""
    P = [_P1(x[..., i], s) for i in range(3)]
    dP = [_g1(x[..., i], s) - _g1(x[..., i] - 1.0, s) for i in range(3)]
    return np.stack([dP[0] * P[1] * P[2], P[0] * dP[1] * P[2], P[0] * P[1] * dP[2]], axis=-1)


def _time_int(f, a, b, n=16):
    """int_a^b f(s) ds with s = u^2 substitution (integrable s^{-1/2} at 0)."""
    xg, wg = np.polynomial.legendre.leggauss(n)
    ua, ub = math.sqrt(a), math.sqrt(b)
    tot = 0.0
    # graded pieces in u towards ua
    edges = ua + (ub - ua) * np.concatenate([[0.0], 0.5 ** np.arange(8, -1, -1.0)])
    for lo, hi in zip(edges[:-1], edges[1:]):
        uu = lo + (hi - lo) * 0.5 * (xg + 1.0)
        for ui, wi in zip(uu, wg):
            tot = tot + 0.5 * (hi - lo) * wi * 2.0 * ui * f(ui * ui)
    return tot


def test_d2_row_sums_divergence_theorem(orc, cube3d):
    nodes, tris, T, n_steps, D2 = (cube3d["nodes"], cube3d["tris"], cube3d["T"],
                                   cube3d["n_steps"], cube3d["D2"])
    h = T / n_steps
    area, normal = orc.triangle_geometry(nodes, tris)
    S1, S2, W = orc.triangle_rule(8)
    N = len(nodes)
    worst = np.zeros(n_steps)
    exact = np.zeros((n_steps, N))
    for j, t3 in enumerate(tris):
        P = nodes[t3]
        x = P[0] + S1[:, None] * (P[1] - P[0]) + S2[:, None] * (P[2] - P[1])
        lam = np.stack([1.0 - S1, S1 - S2, S2], axis=1)
        for d in range(n_steps):
            if d == 0:
                g = _time_int(lambda s: _gradP(x, s), 0.0, h)
            else:
                g = (_time_int(lambda s: _gradP(x, s), d * h, (d + 1) * h) -
                     _time_int(lambda s: _gradP(x, s), (d - 1) * h, d * h))
            ng = -ALPHA * (g @ normal[j])  # -n_x . grad Q_d at the rule points
            for v in range(3):
                exact[d, t3[v]] += 2.0 * area[j] * np.dot(W, lam[:, v] * ng)
    got = D2.sum(axis=2)
    for d in range(n_steps):
        worst[d] = np.abs(got[d] - exact[d]).max() / np.abs(exact[d]).max()
    # quadrature error of the m = 4 regularised rules and the q = 3 regular
    # rule, as for the K row sums; a wrong weight, sign or level is O(1)
    # (observed 1.2e-4, 1.5e-4, 1.0e-5, 3.9e-6, 1.7e-6)
    assert np.all(worst < np.array([1e-3, 1e-3, 1e-4, 4e-5, 2e-5])), worst
    print("D2 row sums: worst relative deviation per block", worst)


def test_neumann_rhs_against_the_dirichlet_rhs(orc):
    nodes, tris = workloads.cube_mesh(2)
    T, n = 0.8, 4
    E, N = len(tris), len(nodes)
    rng = np.random.default_rng(3)
    K1 = rng.normal(size=(n, E, N))
    hd = rng.normal(size=(1, n, E))
    g = rng.normal(size=(1, n, N))
    area, _ = orc.triangle_geometry(nodes, tris)
    f = orc.neumann_rhs(area, tris, K1, hd, T)
    zero = np.zeros_like(K1)
    half_mass = orc.dirichlet_rhs_p1(area, tris, zero, g, T)      # (1/2 M g)
    Kg_rev = orc.toeplitz_matvec_rect(K1, g[:, ::-1].copy())[:, ::-1]  # R K R g
    lhs = float(np.sum(g * f))
    rhs = float(np.sum(hd * half_mass) - np.sum(hd * Kg_rev))
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(g).sum() * np.abs(f).max()), (lhs, rhs)


def test_p1_error_orthogonality(orc):
    nodes, tris = workloads.cube_mesh(2)
    alpha, T, n = 0.8, 0.5, 3
    src = workloads.point_source((1.4, 0.3, 0.6), t0=-0.05)
    g1 = orc.project_dirichlet_p1(nodes, tris, alpha, T, n, src)
    e0, r0 = orc.dirichlet_error_p1(nodes, tris, alpha, T, n, src, g1)
    rng = np.random.default_rng(9)
    v = rng.normal(size=g1.shape)
    eps = 1e-2
    e1, r1 = orc.dirichlet_error_p1(nodes, tris, alpha, T, n, src, g1 + eps * v)
    area, _ = orc.triangle_geometry(nodes, tris)
    N = len(nodes)
    M = np.zeros((N, N))
    for j, t3 in enumerate(tris):
        for a in range(3):
            for b in range(3):
                M[t3[a], t3[b]] += area[j] / 12.0 * (2.0 if a == b else 1.0)
    vv = (T / n) * sum(v[0, k] @ M @ v[0, k] for k in range(n))
    assert r1 == r0
    assert abs((e1 - e0) - eps ** 2 * vv) <= 1e-8 * eps ** 2 * vv, (e1 - e0, eps ** 2 * vv)


def load_neuconv():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table_neuconv.txt")
    rows = []
    with open(path) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                et, ex, comp, proj, rep = line.split()
                rows.append((int(et), int(ex), float(comp), float(proj), float(rep)))
    return rows


def test_table_neuconv_coarsest_run(orc):
    """Cube (-1,1)^3, 192 triangles, 8 steps, alpha 0.5, source (0,0,1.5):
    D_h from the oracle's V, K1 and D2, the projected Neumann data, the
    forward-substitution solve, the L2(Sigma_h) error of u_h."""
    from concurrent.futures import ThreadPoolExecutor
    n_steps, E, comp, proj, _ = load_neuconv()[0]
    alpha, T = 0.5, 1.0
    src = workloads.point_source((0.0, 0.0, 1.5), t0=0.0)
    nodes, tris = workloads.cube_mesh(int(round(math.sqrt(E / 12))), lo=-1.0, hi=1.0)
    chunks = np.array_split(np.arange(E), 8)
    with ThreadPoolExecutor(8) as ex:
        D2 = sum(ex.map(lambda r: orc.assemble_d2(nodes, tris, alpha, T, n_steps, r), chunks))
    V, _ = orc.assemble(nodes, tris, alpha, T, n_steps)
    K1 = orc.assemble_k1(nodes, tris, alpha, T, n_steps)
    D = orc.assemble_d1(nodes, tris, alpha, V) + D2
    area, _ = orc.triangle_geometry(nodes, tris)
    hd = orc.project_neumann(nodes, tris, alpha, T, n_steps, src)
    u = orc.dirichlet_solve(D, orc.neumann_rhs(area, tris, K1, hd, T))
    e2, r2 = orc.dirichlet_error_p1(nodes, tris, alpha, T, n_steps, src, u)
    err = math.sqrt(e2 / r2)
    assert abs(err - comp) <= 0.02 * comp, err
    g1 = orc.project_dirichlet_p1(nodes, tris, alpha, T, n_steps, src)
    e2, r2 = orc.dirichlet_error_p1(nodes, tris, alpha, T, n_steps, src, g1)
    assert abs(math.sqrt(e2 / r2) - proj) <= 0.05 * proj, math.sqrt(e2 / r2)
