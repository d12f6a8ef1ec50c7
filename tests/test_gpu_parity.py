"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances.  Every block entry is a second difference of time-level sums,
V^d = 2 S_d - S_{d+1} - S_{d-1} (eq. vd) or h S_* - S_1 + S_0 (eq. V0), and the
two sides evaluate the sums with different (equally valid) rounding: erf/exp
of different libraries, another summation order.  The difference of an entry
is therefore bounded by c eps (|S_{d-1}| + 2|S_d| + |S_{d+1}|), which can
exceed 1e-12 |V^d| where the difference cancels (large d, far pairs at small
d).  Per block the test requires
    ||A_gpu^d - A_orc^d||_F <= max(1e-12 ||A_orc^d||_F, 64 eps ||C^d||_F),
C^d the entrywise magnitude above, computed from the oracle's own sums.
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


def gpu_assemble(nodes, tris, alpha, T, n_steps, q=3, m=4, storage=capi.STB_STORE_F64, k=True):
    mesh = capi.Mesh(nodes, tris)
    p = capi.stb_default_params(alpha, T, n_steps, q, m, storage=storage)
    dt = torch.float64 if storage == capi.STB_STORE_F64 else torch.float32
    E = mesh.n_tris
    V = torch.full((n_steps, E, E), float("nan"), dtype=dt, device="cuda")
    K = torch.full((n_steps, E, E), float("nan"), dtype=dt, device="cuda") if k else None
    ws = torch.empty(capi.stb_assemble_workspace_size(mesh, p), dtype=torch.uint8, device="cuda")
    capi.stb_assemble(mesh, p, V, K, ws)
    capi.stb_workspace_status(ws)
    torch.cuda.synchronize()
    return mesh, V.double().cpu().numpy(), (K.double().cpu().numpy() if k else None)


def cond_mag(S, h):
    """[rows, n_steps, E] magnitude of the second-difference terms per entry."""
    A = np.abs(S)
    n_steps = S.shape[1] - 2
    C = np.empty((S.shape[0], n_steps, S.shape[2]))
    C[:, 0] = h * A[:, -1] + A[:, 1] + A[:, 0]
    for d in range(1, n_steps):
        C[:, d] = A[:, d - 1] + 2 * A[:, d] + A[:, d + 1]
    return C


def check_blocks(got, ref, S, h, label, extra_rel=0.0):
    """got/ref: [rows, n_steps, E]; returns the worst ratio error/bound."""
    C = cond_mag(S, h)
    worst = 0.0
    for d in range(ref.shape[1]):
        err = np.linalg.norm(got[:, d] - ref[:, d])
        nrm = np.linalg.norm(ref[:, d])
        bound = max(1e-12 * nrm, 64 * EPS * np.linalg.norm(C[:, d])) + extra_rel * nrm
        assert np.all(np.isfinite(got[:, d])), (label, d)
        assert err <= bound, (label, d, err / max(nrm, 1e-300), bound / max(nrm, 1e-300))
        worst = max(worst, err / bound if bound > 0 else 0.0)
    return worst


def test_c1_blocks_match_oracle():
    """cube, 192 triangles, 16 steps, alpha = 1 (the plain FP64 workload)."""
    wl = workloads.workload("cube192_e16")
    nodes, tris, alpha, T, n = wl["nodes"], wl["tris"], wl["alpha"], wl["T"], wl["n_steps"]
    _, V, K = gpu_assemble(nodes, tris, alpha, T, n)
    E = len(tris)
    Vo, Ko, SV, SK = oracle.assemble_rows(nodes, tris, alpha, T, n, np.arange(E), with_sums=True)
    Vg, Kg = V.transpose(1, 0, 2), K.transpose(1, 0, 2)  # -> [rows][d][j]
    h = T / n
    wv = check_blocks(Vg, Vo, SV, h, "V")
    wk = check_blocks(Kg, Ko, SK, h, "K")
    # well-conditioned blocks meet 1e-12 outright
    rel0 = np.linalg.norm(Vg[:, 0] - Vo[:, 0]) / np.linalg.norm(Vo[:, 0])
    assert rel0 < 1e-12
    print("C1 worst error/bound: V %.3f K %.3f; block-0 rel err %.2e" % (wv, wk, rel0))


@pytest.mark.parametrize("n_face,n_steps,q,m", [(2, 13, 2, 3), (2, 1, 3, 4), (1, 9, 1, 1), (2, 8, 4, 5)])
def test_ragged_orders_and_steps(n_face, n_steps, q, m):
    """E not a multiple of the CTA width, E_t not a multiple of the level
    chunk, the smallest and larger quadrature orders, a single step."""
    nodes, tris = workloads.cube_mesh(n_face)
    alpha, T = 0.7, 0.5
    _, V, K = gpu_assemble(nodes, tris, alpha, T, n_steps, q, m)
    Vo, Ko, SV, SK = oracle.assemble_rows(nodes, tris, alpha, T, n_steps, np.arange(len(tris)), q, m,
                                          with_sums=True)
    h = T / n_steps
    check_blocks(V.transpose(1, 0, 2), Vo, SV, h, "V")
    check_blocks(K.transpose(1, 0, 2), Ko, SK, h, "K")


@pytest.mark.parametrize("nf", [1, 2])
def test_icosphere_all_pair_classes(nf):
    """icosahedron (20 triangles: identical, edge and vertex pairs make up half
    of the ordered pairs) and its 80-triangle refinement."""
    nodes, tris = workloads.icosphere(nf)
    alpha, T, n_steps = 1.3, 0.4, 5
    _, V, K = gpu_assemble(nodes, tris, alpha, T, n_steps)
    Vo, Ko, SV, SK = oracle.assemble_rows(nodes, tris, alpha, T, n_steps, np.arange(len(tris)),
                                          with_sums=True)
    h = T / n_steps
    check_blocks(V.transpose(1, 0, 2), Vo, SV, h, "V")
    check_blocks(K.transpose(1, 0, 2), Ko, SK, h, "K")


def test_v_only_and_f32_storage():
    nodes, tris = workloads.cube_mesh(2)
    alpha, T, n = 1.0, 0.6, 6
    _, V64, _ = gpu_assemble(nodes, tris, alpha, T, n, k=False)
    _, V32, K32 = gpu_assemble(nodes, tris, alpha, T, n, storage=capi.STB_STORE_F32)
    Vo, Ko, SV, SK = oracle.assemble_rows(nodes, tris, alpha, T, n, np.arange(len(tris)), with_sums=True)
    h = T / n
    check_blocks(V64.transpose(1, 0, 2), Vo, SV, h, "V64")
    # storage rounding to FP32 adds at most 2^-24 relative per entry
    check_blocks(V32.transpose(1, 0, 2), Vo, SV, h, "V32", extra_rel=2.0 ** -24)
    check_blocks(K32.transpose(1, 0, 2), Ko, SK, h, "K32", extra_rel=2.0 ** -24)


@pytest.mark.slow
def test_c2_sampled_rows():
    """cube, 3072 triangles, 64 steps, alpha = 0.5: the full-size assembly in
    the launch configuration bench.py times, checked on sampled rows."""
    wl = workloads.workload("cube3072_e64", alpha=0.5)
    nodes, tris, alpha, T, n = wl["nodes"], wl["tris"], wl["alpha"], wl["T"], wl["n_steps"]
    _, V, K = gpu_assemble(nodes, tris, alpha, T, n)
    rows = np.array([0, 1537, 3071])
    Vo, Ko, SV, SK = oracle.assemble_rows(nodes, tris, alpha, T, n, rows, with_sums=True)
    h = T / n
    check_blocks(V[:, rows].transpose(1, 0, 2), Vo, SV, h, "V")
    check_blocks(K[:, rows].transpose(1, 0, 2), Ko, SK, h, "K")
    # symmetry of V over the whole matrix (rule shared by (l,j) and (j,l)):
    # rounding of the second difference, scaled by the conditioning
    # ||C^d|| / ||V^d|| measured on the sampled rows
    C = cond_mag(SV, h)
    for d in (0, 1, 63):
        A = V[d]
        kappa = np.linalg.norm(C[:, d]) / np.linalg.norm(Vo[:, d])
        assert np.linalg.norm(A - A.T) <= 2 * 64 * EPS * kappa * np.linalg.norm(A), d


# ---- mixed precision -----------------------------------------------------------
# Every quadrature point in FP32 with cancellation-free forms (closed forms
# minus their part linear in delta for d = 0, 1; Gauss nodes of the reduced
# time integral of eq. V_d for d >= 2).  Stated bound: relative Frobenius
# error per block <= 2e-6 against the FP64 oracle.
MIXED_BOUND = 2e-6


def gpu_assemble_mixed(nodes, tris, alpha, T, n_steps, storage=capi.STB_STORE_F32, q=3, m=4):
    mesh = capi.Mesh(nodes, tris)
    p = capi.stb_default_params(alpha, T, n_steps, q, m, precision=capi.STB_PREC_MIXED,
                                storage=storage)
    dt = torch.float64 if storage == capi.STB_STORE_F64 else torch.float32
    E = mesh.n_tris
    V = torch.full((n_steps, E, E), float("nan"), dtype=dt, device="cuda")
    K = torch.full((n_steps, E, E), float("nan"), dtype=dt, device="cuda")
    ws = torch.empty(capi.stb_assemble_workspace_size(mesh, p), dtype=torch.uint8, device="cuda")
    capi.stb_assemble(mesh, p, V, K, ws)
    capi.stb_workspace_status(ws)
    torch.cuda.synchronize()
    return V.double().cpu().numpy(), K.double().cpu().numpy()


def block_errors(got, ref):
    """got [n_steps][E][E] (library layout) vs ref [rows][n_steps][E] for all rows."""
    g = got.transpose(1, 0, 2)
    return [np.linalg.norm(g[:, d] - ref[:, d]) / np.linalg.norm(ref[:, d]) for d in range(ref.shape[1])]


def test_mixed_c1_blocks():
    wl = workloads.workload("cube192_e16")
    nodes, tris, alpha, T, n = wl["nodes"], wl["tris"], wl["alpha"], wl["T"], wl["n_steps"]
    Vo, Ko = oracle.assemble_rows(nodes, tris, alpha, T, n, np.arange(len(tris)))
    for storage in (capi.STB_STORE_F32, capi.STB_STORE_F64):
        V, K = gpu_assemble_mixed(nodes, tris, alpha, T, n, storage)
        ev, ek = block_errors(V, Vo), block_errors(K, Ko)
        assert max(ev) < MIXED_BOUND and max(ek) < MIXED_BOUND, (ev, ek)
    print("mixed C1 max block error: V %.2e K %.2e" % (max(ev), max(ek)))


# one to three steps; a partial first chunk; chunks with 4 and 3 time nodes;
# chunks with 2 nodes (d0 >= 98), full and cut by n_steps, also at small alpha
@pytest.mark.parametrize("n_face,n_steps,alpha,T", [(2, 1, 1.0, 0.5), (2, 2, 1.0, 0.5), (2, 3, 0.1, 1.0),
                                                   (2, 13, 10.0, 0.3), (2, 40, 0.5, 2.0),
                                                   (2, 130, 1.0, 2.0), (2, 100, 0.2, 1.0),
                                                   (2, 130, 0.05, 1.0)])
def test_mixed_ragged(n_face, n_steps, alpha, T):
    nodes, tris = workloads.cube_mesh(n_face)
    Vo, Ko = oracle.assemble_rows(nodes, tris, alpha, T, n_steps, np.arange(len(tris)))
    V, K = gpu_assemble_mixed(nodes, tris, alpha, T, n_steps)
    ev, ek = block_errors(V, Vo), block_errors(K, Ko)
    assert max(ev) < MIXED_BOUND and max(ek) < MIXED_BOUND, (ev, ek)
    print("mixed n_steps=%d alpha=%g: max block error V %.2e K %.2e" % (n_steps, alpha, max(ev), max(ek)))


def test_mixed_icosphere():
    nodes, tris = workloads.icosphere(2)
    Vo, Ko = oracle.assemble_rows(nodes, tris, 1.3, 0.4, 5, np.arange(len(tris)))
    V, K = gpu_assemble_mixed(nodes, tris, 1.3, 0.4, 5)
    ev, ek = block_errors(V, Vo), block_errors(K, Ko)
    assert max(ev) < MIXED_BOUND and max(ek) < MIXED_BOUND, (ev, ek)


@pytest.mark.slow
def test_mixed_c2_sampled_rows():
    wl = workloads.workload("cube3072_e64", alpha=0.5)
    nodes, tris, alpha, T, n = wl["nodes"], wl["tris"], wl["alpha"], wl["T"], wl["n_steps"]
    V, K = gpu_assemble_mixed(nodes, tris, alpha, T, n)
    rows = np.array([0, 1537, 3071])
    Vo, Ko = oracle.assemble_rows(nodes, tris, alpha, T, n, rows)
    ev = [np.linalg.norm(V[d, rows] - Vo[:, d]) / np.linalg.norm(Vo[:, d]) for d in range(n)]
    ek = [np.linalg.norm(K[d, rows] - Ko[:, d]) / np.linalg.norm(Ko[:, d]) for d in range(n)]
    assert max(ev) < MIXED_BOUND and max(ek) < MIXED_BOUND, (max(ev), max(ek))
    print("mixed C2 rows max block error: V %.2e K %.2e" % (max(ev), max(ek)))


def test_toeplitz_matvec_vs_oracle():
    rng = np.random.default_rng(7)
    E, n_steps, nrhs = 150, 11, 3
    A = rng.normal(size=(n_steps, E, E))
    x = rng.normal(size=(nrhs, n_steps, E))
    y0 = rng.normal(size=(nrhs, n_steps, E))
    ref = oracle.toeplitz_matvec(A, x)
    for storage, dt in ((capi.STB_STORE_F64, torch.float64), (capi.STB_STORE_F32, torch.float32)):
        Ad = torch.tensor(A, dtype=dt, device="cuda")
        Aref = Ad.double().cpu().numpy()
        refs = oracle.toeplitz_matvec(Aref, x) if storage == capi.STB_STORE_F32 else ref
        xd = torch.tensor(x, device="cuda")
        yd = torch.tensor(y0, device="cuda")
        ws = torch.empty(capi.stb_toeplitz_workspace_size(E, n_steps, nrhs), dtype=torch.uint8,
                         device="cuda")
        capi.stb_toeplitz_matvec(Ad, storage, E, n_steps, nrhs, xd, 0.5, yd, ws)
        got = yd.cpu().numpy()
        expect = 0.5 * y0 + refs
        scale = np.abs(Aref).max() * np.abs(x).max() * E * n_steps
        assert np.abs(got - expect).max() <= 4 * EPS * scale


def _matvec_ex(A32, x, y0, beta, arith):
    n_steps, E = A32.shape[0], A32.shape[1]
    nrhs = x.shape[0]
    Ad = torch.tensor(A32, dtype=torch.float32, device="cuda")
    xd = torch.tensor(x, device="cuda")
    yd = torch.tensor(y0, device="cuda")
    ws = torch.empty(capi.stb_toeplitz_ex_workspace_size(E, n_steps, nrhs, arith), dtype=torch.uint8,
                     device="cuda")
    capi.stb_toeplitz_matvec_ex(Ad, capi.STB_STORE_F32, E, n_steps, nrhs, xd, beta, yd, arith, ws)
    capi.stb_workspace_status(ws)
    return yd.cpu().numpy()


# (E, n_steps, nrhs): one 64-column box; two time tiles with a ragged tail;
# three right-hand sides (boxes of two, one unused); five right-hand sides
# (boxes of four, a partly used second group); rows not a multiple of 128
@pytest.mark.parametrize("E,n_steps,nrhs", [(256, 16, 1), (200, 70, 1), (200, 11, 3), (132, 9, 5),
                                            (388, 130, 2)])
def test_toeplitz_matvec_tf32_tensor_cores(E, n_steps, nrhs):
    """tcgen05 TF32 product: blocks read as TF32 (10 stored mantissa bits,
    truncated or rounded: relative error <= 2^-10), x rounded to TF32
    (<= 2^-11), FP32 accumulation (<= K 2^-23 with any rounding of the adder):
    |y - y_exact| <= (2^-10 + 2^-10 + K 2^-23) sum_d |A^d| |x^{k-d}|, K = E (k+1)
    terms."""
    rng = np.random.default_rng(11)
    A = rng.normal(size=(n_steps, E, E)).astype(np.float32).astype(np.float64)
    x = rng.normal(size=(nrhs, n_steps, E))
    y0 = rng.normal(size=(nrhs, n_steps, E))
    got = _matvec_ex(A, x, y0, -0.75, capi.STB_ARITH_TF32)
    exact = -0.75 * y0 + oracle.toeplitz_matvec(A, x)
    mag = oracle.toeplitz_matvec(np.abs(A), np.abs(x))
    K = E * (np.arange(n_steps) + 1.0)
    bound = (2.0 ** -10 + 2.0 ** -10 + K[None, :, None] * 2.0 ** -23) * mag + 1e-14 * np.abs(y0)
    err = np.abs(got - exact)
    assert np.all(err <= bound), float((err / bound).max())
    rel = np.linalg.norm(got - exact) / np.linalg.norm(exact)
    assert rel < 2e-3, rel
    print("TF32 matvec E=%d n=%d nrhs=%d: rel error %.2e, worst err/bound %.2f"
          % (E, n_steps, nrhs, rel, (err / bound).max()))


def test_toeplitz_matvec_double_float():
    """FP32 blocks in FP32-pair arithmetic: exact products, two-float split of
    x (about 48 bits), error-free sums: far below FP32 rounding."""
    rng = np.random.default_rng(12)
    E, n_steps, nrhs = 150, 13, 2
    A = rng.normal(size=(n_steps, E, E)).astype(np.float32).astype(np.float64)
    x = rng.normal(size=(nrhs, n_steps, E))
    y0 = rng.normal(size=(nrhs, n_steps, E))
    got = _matvec_ex(A, x, y0, 2.0, capi.STB_ARITH_DF)
    exact = 2.0 * y0 + oracle.toeplitz_matvec(A, x)
    mag = oracle.toeplitz_matvec(np.abs(A), np.abs(x)) + 2.0 * np.abs(y0)
    err = np.abs(got - exact)
    assert np.all(err <= 2.0 ** -40 * mag), float((err / mag).max())


def test_toeplitz_matvec_ex_rejects():
    E, n_steps = 150, 4  # E not a multiple of 4: no TF32 tensor maps
    A = torch.zeros((n_steps, E, E), dtype=torch.float32, device="cuda")
    x = torch.zeros((1, n_steps, E), dtype=torch.float64, device="cuda")
    ws = torch.empty(capi.stb_toeplitz_ex_workspace_size(E, n_steps, 1, capi.STB_ARITH_TF32),
                     dtype=torch.uint8, device="cuda")
    with pytest.raises(capi.StbError) as e:
        capi.stb_toeplitz_matvec_ex(A, capi.STB_STORE_F32, E, n_steps, 1, x, 0.0, x.clone(),
                                    capi.STB_ARITH_TF32, ws)
    assert e.value.code == -1
    A64 = torch.zeros((n_steps, 152, 152), dtype=torch.float64, device="cuda")
    with pytest.raises(capi.StbError):
        capi.stb_toeplitz_matvec_ex(A64, capi.STB_STORE_F64, 152, n_steps, 1, x, 0.0, x.clone(),
                                    capi.STB_ARITH_DF, ws)
    with pytest.raises(capi.StbError):
        capi.stb_toeplitz_ex_workspace_size(E, n_steps, 1, 7)


@pytest.fixture(scope="module")
def c1_problem():
    wl = workloads.workload("cube192_e16")
    nodes, tris, alpha, T, n = wl["nodes"], wl["tris"], wl["alpha"], wl["T"], wl["n_steps"]
    Vo, Ko = oracle.assemble(nodes, tris, alpha, T, n)
    return dict(wl=wl, Vo=Vo, Ko=Ko)


def test_projection_rhs_solve_error_vs_oracle(c1_problem):
    wl = c1_problem["wl"]
    nodes, tris, alpha, T, n, src = (wl["nodes"], wl["tris"], wl["alpha"], wl["T"], wl["n_steps"],
                                     wl["sources"])
    Vo, Ko = c1_problem["Vo"], c1_problem["Ko"]
    prob = pipeline.DirichletProblem(nodes, tris, alpha, T, n, src)
    # projection
    prob.project()
    go = oracle.project_dirichlet(nodes, tris, alpha, T, n, src)
    g = prob.g.cpu().numpy()
    assert np.abs(g - go).max() <= 1e-13 * np.abs(go).max()
    # right-hand side from the oracle's K and g
    prob.K.copy_(torch.tensor(Ko))
    prob.g.copy_(torch.tensor(go))
    prob.rhs()
    area, _ = oracle.triangle_geometry(nodes, tris)
    fo = oracle.dirichlet_rhs(area, Ko, go, T)
    f = prob.f.cpu().numpy()
    assert np.abs(f - fo).max() <= 1e-13 * np.abs(fo).max() + 64 * EPS * np.abs(go).max() * np.abs(Ko).sum(axis=(0, 2)).max()
    # solve from the oracle's V and f
    prob.V.copy_(torch.tensor(Vo))
    prob.f.copy_(torch.tensor(fo))
    prob.solve()
    wo = oracle.dirichlet_solve(Vo, fo)
    w = prob.w.cpu().numpy()
    # forward error of two backward-stable solves: a small multiple of
    # cond(V_h) eps, V_h the full lower block-triangular matrix
    E = len(tris)
    M = np.zeros((n * E, n * E))
    for k in range(n):
        for i in range(k + 1):
            M[k * E:(k + 1) * E, i * E:(i + 1) * E] = Vo[k - i]
    kappa = np.linalg.cond(M)
    rel = np.linalg.norm(w - wo) / np.linalg.norm(wo)
    assert rel <= 16 * kappa * EPS, (rel, kappa)
    # error norm of the same w
    prob.w.copy_(torch.tensor(wo))
    prob.error()
    e2, r2 = oracle.neumann_error(nodes, tris, alpha, T, n, src, wo)
    out = prob.err.cpu().numpy()
    assert abs(out[0] - e2) <= 1e-12 * r2 and abs(out[1] - r2) <= 1e-12 * r2
    print("C1 solve: rel diff %.2e, cond(V_h) %.2e" % (rel, kappa))


def test_full_pipeline_matches_oracle_pipeline(c1_problem):
    wl = c1_problem["wl"]
    nodes, tris, alpha, T, n, src = (wl["nodes"], wl["tris"], wl["alpha"], wl["T"], wl["n_steps"],
                                     wl["sources"])
    Vo, Ko = c1_problem["Vo"], c1_problem["Ko"]
    prob = pipeline.DirichletProblem(nodes, tris, alpha, T, n, src)
    n0 = capi.stb_launch_count()
    prob.run()
    torch.cuda.synchronize()
    assert capi.stb_launch_count() > n0
    area, _ = oracle.triangle_geometry(nodes, tris)
    go = oracle.project_dirichlet(nodes, tris, alpha, T, n, src)
    wo = oracle.dirichlet_solve(Vo, oracle.dirichlet_rhs(area, Ko, go, T))
    w = prob.w.cpu().numpy()
    assert np.linalg.norm(w - wo) / np.linalg.norm(wo) < 1e-8
    e2, r2 = oracle.neumann_error(nodes, tris, alpha, T, n, src, wo)
    assert abs(prob.relative_error() - math.sqrt(e2 / r2)) < 1e-8


def test_mixed_projection_and_rhs(c1_problem):
    """Mixed precision: data projection in FP32 arithmetic (relative error of
    a few FP32 ulps per element mean); right-hand side with the stored FP32 K
    in double-float arithmetic (as accurate as FP64 up to ~2^-44)."""
    wl = c1_problem["wl"]
    nodes, tris, alpha, T, n, src = (wl["nodes"], wl["tris"], wl["alpha"], wl["T"], wl["n_steps"],
                                     wl["sources"])
    prob = pipeline.DirichletProblem(nodes, tris, alpha, T, n, src, precision=capi.STB_PREC_MIXED,
                                     storage=capi.STB_STORE_F32)
    prob.project()
    go = oracle.project_dirichlet(nodes, tris, alpha, T, n, src)
    g = prob.g.cpu().numpy()
    assert np.abs(g - go).max() <= 1e-5 * np.abs(go).max()
    prob.assemble()
    prob.g.copy_(torch.tensor(go))
    prob.rhs()
    area, _ = oracle.triangle_geometry(nodes, tris)
    K32 = prob.K.double().cpu().numpy()
    fo = oracle.dirichlet_rhs(area, K32, go, T)
    f = prob.f.cpu().numpy()
    assert np.linalg.norm(f - fo) <= 1e-12 * np.linalg.norm(fo)


def test_mixed_solve_refines_to_the_fp32_system(c1_problem):
    """Mixed precision: FP32 factorisation and march, refined with a
    double-float residual until ||f - V_h w|| <= 1e-10 ||f||.  The result must
    solve the stored (FP32) system -- all of it: FP32 rounding leaves the
    stored V^0 symmetric only to ~1e-7, so the reference is the FP64 residual
    of the full block system and its dense FP64 solve (difference bounded by
    cond(V_h) times the residual)."""
    wl = c1_problem["wl"]
    nodes, tris, alpha, T, n, src = (wl["nodes"], wl["tris"], wl["alpha"], wl["T"], wl["n_steps"],
                                     wl["sources"])
    prob = pipeline.DirichletProblem(nodes, tris, alpha, T, n, src, precision=capi.STB_PREC_MIXED,
                                     storage=capi.STB_STORE_F32)
    prob.assemble()
    prob.project()
    prob.rhs()
    prob.solve()
    it, res = capi.stb_solve_report(prob.ws_solve)
    assert 1 <= it <= 8 and res <= 1e-10, (it, res)
    V32 = prob.V.double().cpu().numpy()
    f = prob.f.cpu().numpy()
    w = prob.w.cpu().numpy()
    r64 = f - oracle.toeplitz_matvec(V32, w)
    res64 = np.linalg.norm(r64) / np.linalg.norm(f)
    assert res64 <= 2e-10, res64
    E = len(tris)
    M = np.zeros((n * E, n * E))
    for k in range(n):
        for i in range(k + 1):
            M[k * E:(k + 1) * E, i * E:(i + 1) * E] = V32[k - i]
    wo = np.linalg.solve(M, f[0].reshape(-1))
    kappa = np.linalg.cond(M)
    rel = np.linalg.norm(w[0].reshape(-1) - wo) / np.linalg.norm(wo)
    assert rel <= 4 * kappa * 2e-10, (rel, kappa)
    print("mixed solve: %d refinements, residual %.2e (FP64 recheck %.2e), |w - w_dense|/|w| %.2e, "
          "cond %.1f" % (it, res, res64, rel, kappa))


def _split_first_triangle(nodes, tris):
    """Split triangle 0 at its centroid into three (coplanar, conforming):
    E = 12 n^2 + 2, which is not a multiple of 4."""
    a, b, c = tris[0]
    m = len(nodes)
    nodes = np.vstack([nodes, nodes[[a, b, c]].mean(axis=0)])
    tris = np.vstack([[[a, b, m], [b, c, m], [c, a, m]], tris[1:]]).astype(np.int32)
    return nodes, tris


def _dense_block_system(V, n, E):
    M = np.zeros((n * E, n * E))
    for k in range(n):
        for i in range(k + 1):
            M[k * E:(k + 1) * E, i * E:(i + 1) * E] = V[k - i]
    return M


@pytest.mark.parametrize("split,n_steps,nrhs", [(False, 19, 3), (True, 19, 3), (True, 9, 1)])
def test_solve_panels_rhs_groups_ragged_rows(split, n_steps, nrhs):
    """Forward substitution with ragged time panels (n_steps not a multiple of
    the panel width 8), several right-hand sides (rhs groups of the far-history
    kernel), and E = 194 (no vector loads) against E = 192: FP64 solve versus
    the dense FP64 solve; mixed solve (FP32 blocks) by its FP64 residual."""
    nodes, tris = workloads.cube_mesh(4)
    if split:
        nodes, tris = _split_first_triangle(nodes, tris)
    E = len(tris)
    alpha, T = 0.8, 0.7
    rng = np.random.default_rng(21)
    f = rng.normal(size=(nrhs, n_steps, E))
    for precision, storage in ((capi.STB_PREC_FP64, capi.STB_STORE_F64),
                               (capi.STB_PREC_MIXED, capi.STB_STORE_F32)):
        mesh = capi.Mesh(nodes, tris)
        p = capi.stb_default_params(alpha, T, n_steps, precision=precision, storage=storage)
        dt = torch.float64 if storage == capi.STB_STORE_F64 else torch.float32
        V = torch.empty((n_steps, E, E), dtype=dt, device="cuda")
        ws = torch.empty(capi.stb_assemble_workspace_size(mesh, p), dtype=torch.uint8, device="cuda")
        capi.stb_assemble(mesh, p, V, None, ws)
        fd = torch.tensor(f, device="cuda")
        wd = torch.empty_like(fd)
        wss = torch.empty(capi.stb_solve_workspace_size(mesh, p, nrhs), dtype=torch.uint8,
                          device="cuda")
        capi.stb_dirichlet_solve(mesh, p, V, fd, nrhs, wd, wss)
        w = wd.cpu().numpy()
        Vh = V.double().cpu().numpy()
        r64 = f - oracle.toeplitz_matvec(Vh, w)
        res = np.linalg.norm(r64) / np.linalg.norm(f)
        if precision == capi.STB_PREC_FP64:
            M = _dense_block_system(Vh, n_steps, E)
            kappa = np.linalg.cond(M)
            wo = np.linalg.solve(M, f.reshape(nrhs, -1).T).T.reshape(nrhs, n_steps, E)
            rel = np.linalg.norm(w - wo) / np.linalg.norm(wo)
            assert rel <= 16 * kappa * EPS, (rel, kappa)
            assert res <= 64 * kappa * EPS, res
        else:
            it, rep = capi.stb_solve_report(wss)
            assert 1 <= it <= 8 and rep <= 1e-10, (it, rep)
            assert res <= 2e-10, res
        print("solve E=%d n=%d nrhs=%d prec=%d: residual %.2e cond %.1f"
              % (E, n_steps, nrhs, precision, res, kappa))


def test_not_spd_is_reported():
    nodes, tris = workloads.cube_mesh(1)
    mesh = capi.Mesh(nodes, tris)
    p = capi.stb_default_params(1.0, 1.0, 3)
    E = mesh.n_tris
    V = torch.eye(E, dtype=torch.float64, device="cuda").repeat(3, 1, 1)
    V[0, 5, 5] = -1.0
    f = torch.ones((1, 3, E), dtype=torch.float64, device="cuda")
    w = torch.empty_like(f)
    ws = torch.empty(capi.stb_solve_workspace_size(mesh, p, 1), dtype=torch.uint8, device="cuda")
    with pytest.raises(capi.StbError) as ei:
        capi.stb_dirichlet_solve(mesh, p, V, f, 1, w, ws)
    assert ei.value.code == -5


def test_workspace_errors():
    nodes, tris = workloads.cube_mesh(1)
    mesh = capi.Mesh(nodes, tris)
    p = capi.stb_default_params(1.0, 1.0, 3)
    E = mesh.n_tris
    V = torch.empty((3, E, E), dtype=torch.float64, device="cuda")
    need = capi.stb_assemble_workspace_size(mesh, p)
    small = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(capi.StbError) as ei:
        capi.stb_assemble(mesh, p, V, None, small)
    assert ei.value.code == -8
    big = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    with pytest.raises(capi.StbError) as ei:
        capi.stb_assemble(mesh, p, V, None, big[1:need + 1])  # misaligned view
    assert ei.value.code == -8
