"""GPU parity of the piecewise-linear trial space (Sec. 3.2: the double layer
K_h with nodal hat trial functions of X_h^{1,0}; Sec. 3.4: the L2 projection
of the Dirichlet datum into X_h^{1,0} and the right-hand side
(1/2 M_h + K_h) g1 with the p0 x p1 mass), through the C ABI, against the
FP64 oracle on the same seeded inputs.

Tolerances.  K1^d[l,i] adds, over the triangles j around node i, second
differences in time of sums weighted by barycentric coordinates; on the
convex test surfaces (cube, sphere) r . n_y keeps one sign over a pair, so
the magnitude of the terms is bounded by the p0 magnitudes C^d[l,j]
(second-difference terms of the oracle's own K sums) summed over the star of
i.  Per block the test requires
    ||K1_gpu^d - K1_orc^d||_F <= max(1e-12 ||K1_orc^d||_F, 64 eps ||C1^d||_F),
C1^d[l,i] = sum_{j ∋ i} C^d[l,j].  FP32 storage adds one FP32 rounding per
contribution: 1e-6 relative per block.
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


def _mesh(name):
    if name == "cube2":
        return workloads.cube_mesh(2)
    if name == "cube4":
        return workloads.cube_mesh(4)
    if name == "ico3":
        return workloads.icosphere(3)
    raise KeyError(name)


def _incidence(tris, N):
    inc = np.zeros((len(tris), N))
    for j, t in enumerate(tris):
        inc[j, t] = 1.0
    return inc


def gpu_k1(nodes, tris, alpha, T, n_steps, q=3, m=4, storage=capi.STB_STORE_F64):
    mesh = capi.Mesh(nodes, tris)
    p = capi.stb_default_params(alpha, T, n_steps, q, m, storage=storage)
    dt = torch.float64 if storage == capi.STB_STORE_F64 else torch.float32
    K1 = torch.full((n_steps, mesh.n_tris, mesh.n_nodes), float("nan"), dtype=dt, device="cuda")
    ws = torch.empty(capi.stb_assemble_k1_workspace_size(mesh, p), dtype=torch.uint8, device="cuda")
    capi.stb_assemble_k1(mesh, p, K1, ws)
    capi.stb_workspace_status(ws)
    torch.cuda.synchronize()
    return K1.double().cpu().numpy()


def _cond_k1(SK, h, inc):
    """[rows, n_steps, N]: p0 second-difference magnitudes summed over stars."""
    A = np.abs(SK)
    n_steps = SK.shape[1] - 2
    C = np.empty((SK.shape[0], n_steps, SK.shape[2]))
    C[:, 0] = h * A[:, -1] + A[:, 1] + A[:, 0]
    for d in range(1, n_steps):
        C[:, d] = A[:, d - 1] + 2 * A[:, d] + A[:, d + 1]
    return C @ inc


@pytest.mark.parametrize("name,n_steps,alpha,T", [("cube2", 6, 1.0, 0.6), ("cube4", 9, 0.7, 1.0),
                                                  ("ico3", 17, 2.0, 0.5)])
def test_k1_blocks_match_oracle(name, n_steps, alpha, T):
    """Every row; 6 / 9 / 17 steps are ragged against the 8-step chunks,
    cube4 (192 triangles) spans two CTA column blocks with a ragged tail,
    the sphere has vertex and edge pairs in every orientation."""
    nodes, tris = _mesh(name)
    E, N, h = len(tris), len(nodes), T / n_steps
    got = gpu_k1(nodes, tris, alpha, T, n_steps).transpose(1, 0, 2)  # [E, n_steps, N]
    ref = oracle.assemble_k1_rows(nodes, tris, alpha, T, n_steps, np.arange(E))
    _, _, _, SK = oracle.assemble_rows(nodes, tris, alpha, T, n_steps, np.arange(E),
                                       with_sums=True)
    C1 = _cond_k1(SK, h, _incidence(tris, N))
    worst = 0.0
    for d in range(n_steps):
        assert np.all(np.isfinite(got[:, d])), d
        err, nrm = np.linalg.norm(got[:, d] - ref[:, d]), np.linalg.norm(ref[:, d])
        bound = max(1e-12 * nrm, 64 * EPS * np.linalg.norm(C1[:, d]))
        assert err <= bound, (d, err / nrm, bound / nrm)
        worst = max(worst, err / nrm)
    print("%s: K1 max block rel err %.2e" % (name, worst))


def test_k1_f32_storage_and_quadrature_orders():
    nodes, tris = _mesh("cube4")
    alpha, T, n_steps, q, m = 0.5, 1.0, 5, 4, 3
    E = len(tris)
    got = gpu_k1(nodes, tris, alpha, T, n_steps, q, m, capi.STB_STORE_F32).transpose(1, 0, 2)
    ref = oracle.assemble_k1_rows(nodes, tris, alpha, T, n_steps, np.arange(E), q, m)
    for d in range(n_steps):
        rel = np.linalg.norm(got[:, d] - ref[:, d]) / np.linalg.norm(ref[:, d])
        assert rel <= 1e-6, (d, rel)


MIXED_BOUND = 2e-6


def gpu_k1_mixed(nodes, tris, alpha, T, n_steps, q=3, m=4):
    mesh = capi.Mesh(nodes, tris)
    p = capi.stb_default_params(alpha, T, n_steps, q, m, precision=capi.STB_PREC_MIXED,
                                storage=capi.STB_STORE_F32)
    K1 = torch.full((n_steps, mesh.n_tris, mesh.n_nodes), float("nan"), dtype=torch.float32,
                    device="cuda")
    ws = torch.empty(capi.stb_assemble_k1_workspace_size(mesh, p), dtype=torch.uint8, device="cuda")
    capi.stb_assemble_k1(mesh, p, K1, ws)
    capi.stb_workspace_status(ws)
    torch.cuda.synchronize()
    return K1.double().cpu().numpy()


@pytest.mark.parametrize("name,n_steps,alpha,T", [("cube2", 6, 1.0, 0.6), ("cube4", 9, 0.7, 1.0),
                                                  ("ico3", 17, 2.0, 0.5), ("cube2", 40, 1.0, 1.0),
                                                  ("cube2", 130, 1.0, 2.0), ("ico3", 100, 0.2, 1.0)])
def test_k1_mixed_blocks_match_oracle(name, n_steps, alpha, T):
    """Mixed precision (FP32 points, the cancellation-free time forms of the
    p0 mixed path, FP32 atomics): every row, per block relative Frobenius
    error within the stated mixed bound 2e-6; 40 steps end in a ragged
    sub-chunk, 100 / 130 steps reach the 3- and 2-node chunks."""
    nodes, tris = _mesh(name)
    E = len(tris)
    got = gpu_k1_mixed(nodes, tris, alpha, T, n_steps).transpose(1, 0, 2)
    ref = oracle.assemble_k1_rows(nodes, tris, alpha, T, n_steps, np.arange(E))
    worst = 0.0
    for d in range(n_steps):
        assert np.all(np.isfinite(got[:, d])), d
        rel = np.linalg.norm(got[:, d] - ref[:, d]) / np.linalg.norm(ref[:, d])
        assert rel <= MIXED_BOUND, (d, rel)
        worst = max(worst, rel)
    print("%s, %d steps: mixed K1 max block rel err %.2e" % (name, n_steps, worst))


def test_k1_partition_of_unity_at_full_size():
    """Property at any size: the hat functions sum to one, so sum_i K1^d[l,i]
    equals the row sum of the p0 block K^d (the same rules; 3072 triangles,
    16 steps)."""
    wl = workloads.workload("cube3072_e16")
    nodes, tris, alpha, T, n = wl["nodes"], wl["tris"], wl["alpha"], wl["T"], wl["n_steps"]
    mesh = capi.Mesh(nodes, tris)
    p = capi.stb_default_params(alpha, T, n)
    E, N = mesh.n_tris, mesh.n_nodes
    K1 = torch.empty((n, E, N), dtype=torch.float64, device="cuda")
    ws = torch.empty(capi.stb_assemble_k1_workspace_size(mesh, p), dtype=torch.uint8, device="cuda")
    capi.stb_assemble_k1(mesh, p, K1, ws)
    capi.stb_workspace_status(ws)
    l = 1234
    got = K1[:, l].cpu().numpy()
    s1 = K1.sum(dim=2)
    K1.abs_()
    a1 = K1.sum(dim=2)
    del K1, ws
    V = torch.empty((n, E, E), dtype=torch.float64, device="cuda")
    K = torch.empty((n, E, E), dtype=torch.float64, device="cuda")
    ws = torch.empty(capi.stb_assemble_workspace_size(mesh, p), dtype=torch.uint8, device="cuda")
    capi.stb_assemble(mesh, p, V, K, ws)
    capi.stb_workspace_status(ws)
    s0 = K.sum(dim=2)
    del V, K, ws
    dev = (s1 - s0).abs() / a1
    assert float(dev.max()) <= 1e-11, float(dev.max())
    # and one sampled row against the oracle
    ro = oracle.assemble_k1_rows(nodes, tris, alpha, T, n, np.array([l]))[0]
    for d in range(n):
        assert np.linalg.norm(got[d] - ro[d]) <= 1e-10 * np.linalg.norm(ro[d]), d


def test_k1_mixed_at_full_size():
    """The bench workload (cube, 3072 triangles, 64 steps, alpha 0.5) in
    mixed precision: three sampled rows against the oracle (stated bound),
    and for every row the partition of unity against the mixed p0 K of the
    same rules (1e-5 of sum |K1|: two FP32 evaluations of the same sums)."""
    wl = workloads.workload("cube3072_e64")
    nodes, tris, T, n = wl["nodes"], wl["tris"], wl["T"], wl["n_steps"]
    alpha = 0.5
    mesh = capi.Mesh(nodes, tris)
    p = capi.stb_default_params(alpha, T, n, precision=capi.STB_PREC_MIXED,
                                storage=capi.STB_STORE_F32)
    E, N = mesh.n_tris, mesh.n_nodes
    K1 = torch.empty((n, E, N), dtype=torch.float32, device="cuda")
    ws = torch.empty(capi.stb_assemble_k1_workspace_size(mesh, p), dtype=torch.uint8, device="cuda")
    capi.stb_assemble_k1(mesh, p, K1, ws)
    capi.stb_workspace_status(ws)
    rows = [0, 1537, 3071]
    got = K1[:, rows].double().cpu().numpy()
    s1 = K1.double().sum(dim=2)
    a1 = K1.double().abs().sum(dim=2)
    del K1, ws
    V = torch.empty((n, E, E), dtype=torch.float32, device="cuda")
    K = torch.empty((n, E, E), dtype=torch.float32, device="cuda")
    ws = torch.empty(capi.stb_assemble_workspace_size(mesh, p), dtype=torch.uint8, device="cuda")
    capi.stb_assemble(mesh, p, V, K, ws)
    capi.stb_workspace_status(ws)
    s0 = K.double().sum(dim=2)
    del V, K, ws
    torch.cuda.empty_cache()
    dev = float(((s1 - s0).abs() / a1).max())
    assert dev <= 1e-5, dev
    ref = oracle.assemble_k1_rows(nodes, tris, alpha, T, n, np.array(rows))
    for i in range(len(rows)):
        for d in range(n):
            rel = np.linalg.norm(got[d, i] - ref[i, d]) / np.linalg.norm(ref[i, d])
            assert rel <= MIXED_BOUND, (rows[i], d, rel)
    print("mixed K1 at 3072 x 64: partition of unity %.2e" % dev)


@pytest.mark.parametrize("name,n_steps", [("cube2", 3), ("cube4", 16), ("ico3", 7)])
@pytest.mark.parametrize("precision", [capi.STB_PREC_FP64, capi.STB_PREC_MIXED])
def test_projection_p1_matches_oracle(name, n_steps, precision):
    nodes, tris = _mesh(name)
    alpha, T = 0.8, 0.5
    src = workloads.random_sources(np.random.default_rng(11), 2, n_src=2, t0=-0.05)
    mesh = capi.Mesh(nodes, tris)
    p = capi.stb_default_params(alpha, T, n_steps, precision=precision)
    g1 = torch.full((2, n_steps, mesh.n_nodes), float("nan"), dtype=torch.float64, device="cuda")
    ws = torch.empty(capi.stb_project_p1_workspace_size(mesh, p, 2, 2), dtype=torch.uint8,
                     device="cuda")
    capi.stb_project_dirichlet_p1(mesh, p, src, g1, ws)
    capi.stb_workspace_status(ws)
    ref = oracle.project_dirichlet_p1(nodes, tris, alpha, T, n_steps, src)
    got = g1.cpu().numpy()
    tol = 1e-12 if precision == capi.STB_PREC_FP64 else 1e-5
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), np.abs(got - ref).max()


def test_projection_p1_rejects_unused_nodes():
    nodes, tris = workloads.cube_mesh(2)
    nodes = np.vstack([nodes, [[5.0, 5.0, 5.0]]])  # a node in no triangle
    mesh = capi.Mesh(nodes, tris)
    p = capi.stb_default_params(1.0, 1.0, 2)
    with pytest.raises(capi.StbError):
        capi.stb_project_p1_workspace_size(mesh, p, 1, 1)


@pytest.mark.parametrize("storage", [capi.STB_STORE_F64, capi.STB_STORE_F32])
def test_rhs_p1_matches_oracle(storage):
    """From the oracle's K1 and g1: the rectangular block-Toeplitz product
    (192 x 98 blocks, 16 steps: two time tiles, ragged row tiles) and the
    p0 x p1 mass; error bound n eps times the magnitude of the terms."""
    nodes, tris = _mesh("cube4")
    alpha, T, n = 1.0, 1.0, 16
    src = workloads.random_sources(np.random.default_rng(4), 3, t0=-0.1)
    K1 = oracle.assemble_k1(nodes, tris, alpha, T, n)
    if storage == capi.STB_STORE_F32:
        K1 = K1.astype(np.float32).astype(np.float64)
    g1 = oracle.project_dirichlet_p1(nodes, tris, alpha, T, n, src)
    area, _ = oracle.triangle_geometry(nodes, tris)
    fo = oracle.dirichlet_rhs_p1(area, tris, K1, g1, T)
    mag = oracle.dirichlet_rhs_p1(area, tris, np.abs(K1), np.abs(g1), T)
    mesh = capi.Mesh(nodes, tris)
    p = capi.stb_default_params(alpha, T, n, storage=storage)
    dt = torch.float64 if storage == capi.STB_STORE_F64 else torch.float32
    f = torch.full((3, n, len(tris)), float("nan"), dtype=torch.float64, device="cuda")
    ws = torch.empty(capi.stb_rhs_p1_workspace_size(mesh, p, 3), dtype=torch.uint8, device="cuda")
    capi.stb_dirichlet_rhs_p1(mesh, p, torch.tensor(K1, dtype=dt, device="cuda"),
                              torch.tensor(g1, device="cuda"), 3, f, ws)
    capi.stb_workspace_status(ws)
    got = f.cpu().numpy()
    n_terms = n * len(nodes) + 3
    assert np.all(np.abs(got - fo) <= n_terms * EPS * mag + 1e-300)


def test_p1_pipeline_matches_oracle_pipeline():
    """Assembly (V, K1), projection, right-hand side, solve and error on the
    GPU against the oracle's p1 pipeline (cube, 192 triangles, 16 steps)."""
    wl = workloads.workload("cube192_e16")
    nodes, tris, alpha, T, n, src = (wl["nodes"], wl["tris"], wl["alpha"], wl["T"], wl["n_steps"],
                                     wl["sources"])
    prob = pipeline.DirichletProblem(nodes, tris, alpha, T, n, src, data="p1")
    prob.run()
    torch.cuda.synchronize()
    Vo, _ = oracle.assemble(nodes, tris, alpha, T, n)
    K1 = oracle.assemble_k1(nodes, tris, alpha, T, n)
    area, _ = oracle.triangle_geometry(nodes, tris)
    g1 = oracle.project_dirichlet_p1(nodes, tris, alpha, T, n, src)
    wo = oracle.dirichlet_solve(Vo, oracle.dirichlet_rhs_p1(area, tris, K1, g1, T))
    w = prob.w.cpu().numpy()
    assert np.linalg.norm(w - wo) / np.linalg.norm(wo) < 1e-8
    e2, r2 = oracle.neumann_error(nodes, tris, alpha, T, n, src, wo)
    assert abs(prob.relative_error() - math.sqrt(e2 / r2)) < 1e-8
    print("p1 pipeline: L2 error %.4f" % prob.relative_error())


def _dirconv_rows():
    import test_oracle_solve
    return test_oracle_solve.load_dirconv()


@pytest.mark.parametrize("row", [0, 1, 2, pytest.param(3, marks=pytest.mark.slow)])
def test_table_dirconv_p1_on_gpu(row):
    """Table dirconv (cube (-1,1)^3, alpha = 0.5, source (0,0,1.5), T = 1)
    with the paper's piecewise-linear data, every step on the GPU: the
    computed error against the printed one (2 %, as for the oracle: the
    quadrature orders and the diagonal direction of the squares are not
    printed)."""
    n_steps, E, comp, _ = _dirconv_rows()[row]
    nodes, tris = workloads.cube_mesh(int(round(math.sqrt(E / 12))), lo=-1.0, hi=1.0)
    src = workloads.point_source((0.0, 0.0, 1.5), t0=0.0)
    prec = capi.STB_PREC_FP64 if row < 2 else capi.STB_PREC_MIXED
    store = capi.STB_STORE_F64 if row < 2 else capi.STB_STORE_F32
    prob = pipeline.DirichletProblem(nodes, tris, 0.5, 1.0, n_steps, src, data="p1",
                                     precision=prec, storage=store)
    prob.run()
    err = prob.relative_error()
    print("dirconv row %d (E_t %d, E_x %d): computed %.4f, printed %.3g" % (row, n_steps, E, err,
                                                                             comp))
    assert abs(err - comp) < 0.02 * comp, err
