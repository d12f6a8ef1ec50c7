"""GPU parity of the potentials (Sec. 3.5: single-layer potential V~ w_h and
double-layer potential W u_h of the representation formula, eq. repr)
through the C ABI, against the FP64 oracle on the same seeded inputs, and
the paper's printed evaluation errors of the representation formula.

Tolerance.  The oracle forms the paper's differences of antiderivatives
(erf at d h + eps minus erf at (d+1) h + eps), the library one erfc value
per level weighted by backward differences of the density (summation by
parts); both are FP64 rearrangements of the same sum.  Each of the at most
2 (k + 2) antiderivative values of a point carries a rounding error of a
few ulps of its size, at most 1/(4 pi alpha rho) |w| per unit area (single
layer) and |r.n|/(4 pi rho^3) |u| (double layer), so per point
    |gpu - oracle| <= 64 eps (k + 2) M_p,
M_p = sum_j 2 Delta_j max_i |density of j| / (4 pi min(alpha, 1) rho_lo min(1, rho_lo)^2),
rho_lo a lower bound of the distance from x_p to triangle j (the bound covers
both 1/rho and 1/rho^2).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2102_09811_gb300 import capi, pipeline

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module", autouse=True)
def cuda_device():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    capi._library()


def gpu_potentials(nodes, tris, alpha, T, n_steps, pts, w=None, u1=None, q=4,
                   precision=capi.STB_PREC_FP64):
    mesh = capi.Mesh(nodes, tris)
    p = capi.stb_default_params(alpha, T, n_steps, precision=precision)
    nrhs = (w if w is not None else u1).shape[0]
    dev = lambda a: None if a is None else torch.tensor(a, dtype=torch.float64, device="cuda")
    slp = torch.full((nrhs, len(pts)), float("nan"), dtype=torch.float64, device="cuda") \
        if w is not None else None
    dlp = torch.full((nrhs, len(pts)), float("nan"), dtype=torch.float64, device="cuda") \
        if u1 is not None else None
    ws = torch.empty(capi.stb_potentials_workspace_size(mesh, p, nrhs, len(pts), q),
                     dtype=torch.uint8, device="cuda")
    capi.stb_potentials(mesh, p, dev(pts), dev(w), dev(u1), nrhs, slp, dlp, ws, q)
    capi.stb_workspace_status(ws)
    return (None if slp is None else slp.cpu().numpy(), None if dlp is None else dlp.cpu().numpy())


def magnitude(nodes, tris, alpha, T, n_steps, pts, dens_per_tri):
    """M_p of the module docstring; dens_per_tri [E] = max |density| of j."""
    P = nodes[tris]  # [E, 3, 3]
    c = P.mean(axis=1)
    R = np.linalg.norm(P - c[:, None, :], axis=2).max(axis=1)
    area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    M = np.zeros(len(pts))
    for i, x in enumerate(pts):
        lo = np.maximum(np.linalg.norm(x[:3] - c, axis=1) - R, 1e-3)
        M[i] = np.sum(2 * area * dens_per_tri / (4 * np.pi * min(alpha, 1.0) * lo *
                                                 np.minimum(1.0, lo) ** 2))
    h = T / n_steps
    k = np.minimum(np.floor(pts[:, 3] / h), n_steps - 1)
    return M * (k + 2)


def _points(rng, n, T, lo=0.2, hi=0.8):
    x = rng.uniform(lo, hi, size=(n, 3))
    t = rng.uniform(0.0, T, size=(n, 1))
    return np.concatenate([x, t], axis=1)


@pytest.mark.parametrize("n_face,n_steps,q,alpha", [(4, 5, 4, 0.7), (2, 9, 2, 2.0),
                                                    (3, 1, 5, 0.3)])
def test_potentials_match_oracle(n_face, n_steps, q, alpha):
    """Random densities (3 right-hand sides: one pass of 4 and a ragged
    second pass is covered by nrhs = 5 below), random interior points and
    times, plus t = 0, t = T, a step boundary and the first step."""
    nodes, tris = workloads.cube_mesh(n_face)
    T = 0.8
    h = T / n_steps
    rng = np.random.default_rng(n_face * 100 + n_steps)
    E, N = len(tris), len(nodes)
    w = rng.normal(size=(3, n_steps, E))
    u1 = rng.normal(size=(3, n_steps, N))
    pts = np.concatenate([_points(rng, 150, T),
                          [[0.5, 0.5, 0.5, T], [0.4, 0.6, 0.5, 0.0], [0.3, 0.5, 0.6, h],
                           [0.6, 0.4, 0.45, 0.3 * h]]])
    sg, dg = gpu_potentials(nodes, tris, alpha, T, n_steps, pts, w, u1, q)
    so, do = oracle.potentials(nodes, tris, alpha, T, n_steps, pts, w, u1, q)
    Ms = magnitude(nodes, tris, alpha, T, n_steps, pts, np.abs(w).max(axis=(0, 1)))
    Md = magnitude(nodes, tris, alpha, T, n_steps, pts, np.abs(u1).max(axis=(0, 1))[tris].max(axis=1))
    assert np.all(np.isfinite(sg)) and np.all(np.isfinite(dg))
    assert np.all(np.abs(sg - so) <= 64 * EPS * Ms), np.max(np.abs(sg - so) / Ms)
    assert np.all(np.abs(dg - do) <= 64 * EPS * Md), np.max(np.abs(dg - do) / Md)
    assert np.all(sg[:, -3] == 0.0) and np.all(dg[:, -3] == 0.0)  # t = 0
    print("potentials: max |diff| / M  slp %.2e  dlp %.2e" %
          (np.max(np.abs(sg - so) / Ms), np.max(np.abs(dg - do) / Md)))


def test_potentials_one_sided_and_many_rhs():
    """Single layer alone, double layer alone, and 5 right-hand sides (two
    passes of the kernel) give the same values as the combined call."""
    nodes, tris = workloads.icosphere(3)
    T, n_steps, alpha = 1.0, 7, 1.0
    rng = np.random.default_rng(5)
    E, N = len(tris), len(nodes)
    w = rng.normal(size=(5, n_steps, E))
    u1 = rng.normal(size=(5, n_steps, N))
    pts = np.concatenate([rng.uniform(-0.4, 0.4, size=(64, 3)), rng.uniform(0, T, size=(64, 1))], 1)
    s_both, d_both = gpu_potentials(nodes, tris, alpha, T, n_steps, pts, w, u1)
    s_only, _ = gpu_potentials(nodes, tris, alpha, T, n_steps, pts, w=w)
    _, d_only = gpu_potentials(nodes, tris, alpha, T, n_steps, pts, u1=u1)
    assert np.array_equal(s_both, s_only) and np.array_equal(d_both, d_only)
    s1, d1 = gpu_potentials(nodes, tris, alpha, T, n_steps, pts, w[4:], u1[4:])
    assert np.array_equal(s1[0], s_both[4]) and np.array_equal(d1[0], d_both[4])


def test_potentials_flag_times_outside_the_interval():
    nodes, tris = workloads.cube_mesh(2)
    mesh = capi.Mesh(nodes, tris)
    p = capi.stb_default_params(1.0, 1.0, 4)
    pts = torch.tensor([[0.5, 0.5, 0.5, 0.5], [0.5, 0.5, 0.5, 1.5]], dtype=torch.float64,
                       device="cuda")
    w = torch.ones((1, 4, len(tris)), dtype=torch.float64, device="cuda")
    slp = torch.empty((1, 2), dtype=torch.float64, device="cuda")
    ws = torch.empty(capi.stb_potentials_workspace_size(mesh, p, 1, 2, 4), dtype=torch.uint8,
                     device="cuda")
    capi.stb_potentials(mesh, p, pts, w, None, 1, slp, None, ws)
    with pytest.raises(capi.StbError):
        capi.stb_workspace_status(ws)
    assert float(slp[0, 1]) == 0.0 and float(slp[0, 0]) > 0.0
    with pytest.raises(capi.StbError):
        capi.stb_potentials_workspace_size(mesh, p, 1, 2, 6)  # q_space > 5


def test_reprsc_workload_sampled_points():
    """The potential workload of Table reprsc at its full size (cube
    (-1,1)^3, 3072 triangles, 32 steps, 33 x 33 points x 32 times = 34848
    points, one right-hand side): every point on the GPU, 48 seeded points
    against the oracle."""
    nodes, tris = workloads.cube_mesh(16, lo=-1.0, hi=1.0)
    T, n_steps, alpha = 1.0, 32, 0.5
    pts = workloads.reprsc_points(n_steps, T)
    assert len(pts) == 34848
    rng = np.random.default_rng(32)
    E, N = len(tris), len(nodes)
    w = rng.normal(size=(1, n_steps, E))
    u1 = rng.normal(size=(1, n_steps, N))
    sg, dg = gpu_potentials(nodes, tris, alpha, T, n_steps, pts, w, u1)
    idx = rng.choice(len(pts), size=48, replace=False)
    so, do = oracle.potentials(nodes, tris, alpha, T, n_steps, pts[idx], w, u1)
    Ms = magnitude(nodes, tris, alpha, T, n_steps, pts[idx], np.abs(w).max(axis=(0, 1)))
    Md = magnitude(nodes, tris, alpha, T, n_steps, pts[idx],
                   np.abs(u1).max(axis=(0, 1))[tris].max(axis=1))
    assert np.all(np.abs(sg[:, idx] - so) <= 64 * EPS * Ms)
    assert np.all(np.abs(dg[:, idx] - do) <= 64 * EPS * Md)


def gpu_potentials_grid(nodes, tris, alpha, T, n_steps, pts3, eps, w=None, u1=None, q=4,
                        precision=capi.STB_PREC_FP64):
    mesh = capi.Mesh(nodes, tris)
    p = capi.stb_default_params(alpha, T, n_steps, precision=precision)
    nrhs = (w if w is not None else u1).shape[0]
    dev = lambda a: None if a is None else torch.tensor(a, dtype=torch.float64, device="cuda")
    shape = (nrhs, n_steps, len(pts3))
    slp = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda") if w is not None else None
    dlp = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda") if u1 is not None else None
    ws = torch.empty(capi.stb_potentials_grid_workspace_size(mesh, p, nrhs, len(pts3), q),
                     dtype=torch.uint8, device="cuda")
    capi.stb_potentials_grid(mesh, p, dev(pts3), eps, dev(w), dev(u1), nrhs, slp, dlp, ws, q)
    capi.stb_workspace_status(ws)
    return (None if slp is None else slp.cpu().numpy(), None if dlp is None else dlp.cpu().numpy())


@pytest.mark.parametrize("n_face,n_steps,eps_frac,nrhs", [(4, 20, 0.5, 2), (3, 7, 0.0, 1),
                                                          (2, 3, 1.0, 5)])
def test_potentials_grid_matches_oracle(n_face, n_steps, eps_frac, nrhs):
    """Fixed points at every t_k + eps (eps = h/2, 0 and h; 20 steps span two
    time tiles of the block-Toeplitz product, 70 points a ragged row tile)
    against the oracle at the same space-time points."""
    nodes, tris = workloads.cube_mesh(n_face)
    T, alpha = 1.0, 0.8
    h = T / n_steps
    eps = eps_frac * h
    rng = np.random.default_rng(n_steps)
    E, N = len(tris), len(nodes)
    w = rng.normal(size=(nrhs, n_steps, E))
    u1 = rng.normal(size=(nrhs, n_steps, N))
    pts3 = rng.uniform(0.2, 0.8, size=(70, 3))
    sg, dg = gpu_potentials_grid(nodes, tris, alpha, T, n_steps, pts3, eps, w, u1)
    pts = np.concatenate([np.concatenate([pts3, np.full((70, 1), k * h + eps)], axis=1)
                          for k in range(n_steps)])
    pts[:, 3] = np.minimum(pts[:, 3], T)
    so, do = oracle.potentials(nodes, tris, alpha, T, n_steps, pts, w, u1)
    Ms = magnitude(nodes, tris, alpha, T, n_steps, pts, np.abs(w).max(axis=(0, 1)))
    Md = magnitude(nodes, tris, alpha, T, n_steps, pts, np.abs(u1).max(axis=(0, 1))[tris].max(axis=1))
    sg, dg = sg.reshape(nrhs, -1), dg.reshape(nrhs, -1)
    assert np.all(np.abs(sg - so) <= 64 * EPS * Ms), np.max(np.abs(sg - so) / Ms)
    assert np.all(np.abs(dg - do) <= 64 * EPS * Md), np.max(np.abs(dg - do) / Md)


def test_potentials_grid_reprsc_matches_direct():
    """The Table reprsc workload (3072 triangles, 32 steps, 1089 points at
    the step midpoints) through both kernels: the level blocks with the
    block-Toeplitz product and the per-point kernel agree to rounding."""
    nodes, tris = workloads.cube_mesh(16, lo=-1.0, hi=1.0)
    T, n_steps, alpha = 1.0, 32, 0.5
    pts = workloads.reprsc_points(n_steps, T)
    rng = np.random.default_rng(33)
    w = rng.normal(size=(1, n_steps, len(tris)))
    u1 = rng.normal(size=(1, n_steps, len(nodes)))
    sd, dd = gpu_potentials(nodes, tris, alpha, T, n_steps, pts, w, u1)
    sg, dg = gpu_potentials_grid(nodes, tris, alpha, T, n_steps, pts[:1089, :3], 0.5 * T / n_steps,
                                 w, u1)
    sg, dg = sg.reshape(1, -1), dg.reshape(1, -1)  # [k][p] = the time-major point order
    assert np.max(np.abs(sg - sd)) <= 1e-11 * np.max(np.abs(sd))
    assert np.max(np.abs(dg - dd)) <= 1e-11 * np.max(np.abs(dd))


# Level blocks from FP32 quadrature points (STB_PREC_MIXED): every level sum
# is a sum of positive terms (erfc, and erfc + 2x exp(-x^2)/sqrt(pi) for the
# double layer), so each level value carries a few FP32 roundings; the
# potentials (double-float products of those values with the density differences)
# are tested at 1e-5 of their largest value.
MIXED_POT = 1e-5


@pytest.mark.parametrize("n_face,n_steps,eps_frac,nrhs", [(4, 20, 0.5, 2), (2, 3, 1.0, 5)])
def test_potentials_grid_mixed_matches_oracle(n_face, n_steps, eps_frac, nrhs):
    nodes, tris = workloads.cube_mesh(n_face)
    T, alpha = 1.0, 0.8
    h = T / n_steps
    eps = eps_frac * h
    rng = np.random.default_rng(n_steps + 1)
    E, N = len(tris), len(nodes)
    w = rng.normal(size=(nrhs, n_steps, E))
    u1 = rng.normal(size=(nrhs, n_steps, N))
    pts3 = rng.uniform(0.2, 0.8, size=(70, 3))
    sg, dg = gpu_potentials_grid(nodes, tris, alpha, T, n_steps, pts3, eps, w, u1,
                                 precision=capi.STB_PREC_MIXED)
    pts = np.concatenate([np.concatenate([pts3, np.full((70, 1), k * h + eps)], axis=1)
                          for k in range(n_steps)])
    pts[:, 3] = np.minimum(pts[:, 3], T)
    so, do = oracle.potentials(nodes, tris, alpha, T, n_steps, pts, w, u1)
    sg, dg = sg.reshape(nrhs, -1), dg.reshape(nrhs, -1)
    es = np.max(np.abs(sg - so)) / np.max(np.abs(so))
    ed = np.max(np.abs(dg - do)) / np.max(np.abs(do))
    assert es <= MIXED_POT and ed <= MIXED_POT, (es, ed)
    print("mixed level blocks: max error / max value %.2e (single), %.2e (double)" % (es, ed))


def test_potentials_mixed_match_oracle():
    """The per-point kernel with FP32 level values (FP64 density sums) at
    arbitrary space-time points, against the oracle."""
    nodes, tris = workloads.cube_mesh(3)
    T, n_steps, alpha = 1.0, 9, 0.6
    rng = np.random.default_rng(19)
    E, N = len(tris), len(nodes)
    w = rng.normal(size=(2, n_steps, E))
    u1 = rng.normal(size=(2, n_steps, N))
    pts = np.concatenate([rng.uniform(0.15, 0.85, size=(60, 3)), rng.uniform(0.0, T, size=(60, 1))],
                         axis=1)
    sg, dg = gpu_potentials(nodes, tris, alpha, T, n_steps, pts, w, u1,
                            precision=capi.STB_PREC_MIXED)
    so, do = oracle.potentials(nodes, tris, alpha, T, n_steps, pts, w, u1)
    es = np.max(np.abs(sg - so)) / np.max(np.abs(so))
    ed = np.max(np.abs(dg - do)) / np.max(np.abs(do))
    assert es <= MIXED_POT and ed <= MIXED_POT, (es, ed)
    print("mixed per-point potentials: max error / max value %.2e (single), %.2e (double)"
          % (es, ed))


def test_potentials_grid_mixed_reprsc():
    """The Table reprsc workload with the mixed level blocks against the
    FP64 level blocks."""
    nodes, tris = workloads.cube_mesh(16, lo=-1.0, hi=1.0)
    T, n_steps, alpha = 1.0, 32, 0.5
    pts3 = workloads.reprsc_points(n_steps, T)[:1089, :3]
    rng = np.random.default_rng(34)
    w = rng.normal(size=(1, n_steps, len(tris)))
    u1 = rng.normal(size=(1, n_steps, len(nodes)))
    s64, d64 = gpu_potentials_grid(nodes, tris, alpha, T, n_steps, pts3, 0.5 * T / n_steps, w, u1)
    s32, d32 = gpu_potentials_grid(nodes, tris, alpha, T, n_steps, pts3, 0.5 * T / n_steps, w, u1,
                                   precision=capi.STB_PREC_MIXED)
    es = np.max(np.abs(s32 - s64)) / np.max(np.abs(s64))
    ed = np.max(np.abs(d32 - d64)) / np.max(np.abs(d64))
    assert es <= MIXED_POT and ed <= MIXED_POT, (es, ed)
    print("reprsc mixed vs FP64 level blocks: %.2e (single), %.2e (double)" % (es, ed))


def _repr_rows():
    import test_oracle_potentials
    return test_oracle_potentials.load_repr_golden(), test_oracle_potentials.repr_points()


@pytest.mark.parametrize("row", [0, 1, 2, pytest.param(3, marks=pytest.mark.slow)])
def test_table_dirconv_representation_on_gpu(row):
    """Table dirconv, representation column (cube (-1,1)^3, alpha = 0.5,
    source (0,0,1.5), p1 data, w_h computed): u_h = V~ w_h - W g_h at the
    10^4 nodes, every step on the GPU, against the printed l2 error (2 %)."""
    import test_oracle_potentials
    rows, pts = _repr_rows()
    n_steps, E, l2 = rows[row]
    nodes, tris = workloads.cube_mesh(int(round(math.sqrt(E / 12))), lo=-1.0, hi=1.0)
    src = workloads.point_source((0.0, 0.0, 1.5), t0=0.0)
    prec = capi.STB_PREC_FP64 if row < 2 else capi.STB_PREC_MIXED
    store = capi.STB_STORE_F64 if row < 2 else capi.STB_STORE_F32
    prob = pipeline.DirichletProblem(nodes, tris, 0.5, 1.0, n_steps, src, data="p1",
                                     precision=prec, storage=store)
    prob.run()
    uh = prob.representation(pts)[0].cpu().numpy()
    ue = test_oracle_potentials.exact_solution(pts)
    err = np.linalg.norm(uh - ue) / np.linalg.norm(ue)
    print("dirconv row %d: representation l2 %.4e, printed %.3g" % (row, err, l2))
    assert abs(err - l2) <= 0.02 * l2, err


@pytest.mark.parametrize("q,nrhs,eps_frac", [(2, 5, 0.0), (5, 1, 1.0)])
def test_potentials_mixed_orders_and_passes(q, nrhs, eps_frac):
    """Mixed potentials at other rule orders, five right-hand sides (two
    passes of the per-point kernel) and eps = 0 / h on the grid form, against
    the oracle at the same points."""
    nodes, tris = workloads.cube_mesh(2)
    T, n_steps, alpha = 0.8, 6, 1.1
    h = T / n_steps
    rng = np.random.default_rng(q * 10 + nrhs)
    w = rng.normal(size=(nrhs, n_steps, len(tris)))
    u1 = rng.normal(size=(nrhs, n_steps, len(nodes)))
    pts = np.concatenate([rng.uniform(0.2, 0.8, size=(25, 3)), rng.uniform(0.0, T, size=(25, 1))],
                         axis=1)
    sg, dg = gpu_potentials(nodes, tris, alpha, T, n_steps, pts, w, u1, q=q,
                            precision=capi.STB_PREC_MIXED)
    so, do = oracle.potentials(nodes, tris, alpha, T, n_steps, pts, w, u1, q=q)
    assert np.max(np.abs(sg - so)) <= MIXED_POT * np.max(np.abs(so))
    assert np.max(np.abs(dg - do)) <= MIXED_POT * np.max(np.abs(do))
    pts3, eps = pts[:, :3], eps_frac * h
    sgg, dgg = gpu_potentials_grid(nodes, tris, alpha, T, n_steps, pts3, eps, w, u1, q=q,
                                   precision=capi.STB_PREC_MIXED)
    pg = np.concatenate([np.concatenate([pts3, np.full((25, 1), min(k * h + eps, T))], axis=1)
                         for k in range(n_steps)])
    sgo, dgo = oracle.potentials(nodes, tris, alpha, T, n_steps, pg, w, u1, q=q)
    sgg, dgg = sgg.reshape(nrhs, -1), dgg.reshape(nrhs, -1)
    assert np.max(np.abs(sgg - sgo)) <= MIXED_POT * np.max(np.abs(sgo))
    assert np.max(np.abs(dgg - dgo)) <= MIXED_POT * np.max(np.abs(dgo))
