"""GPU parity on non-uniform time grids (Sec. 7): the block lower-triangular
assembly, product, forward substitution, data projection, right-hand side and
error through the C ABI against the FP64 oracle on the same inputs.

Tolerance: 1e-10 relative per block for the assembly (four-corner
combinations of the antiderivative cancel like the uniform second
differences, the two sides round differently), the FP64 rounding bounds of
the uniform tests elsewhere."""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2102_09811_gb300 import capi, pipeline

pytestmark = pytest.mark.gpu
GRADED = np.array([0.0, 0.02, 0.05, 0.1, 0.2, 0.35, 0.6])


@pytest.fixture(scope="module", autouse=True)
def cuda_device():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    capi._library()


def gpu_assemble_nu(nodes, tris, alpha, times, precision=capi.STB_PREC_FP64):
    mesh = capi.Mesh(nodes, tris)
    n = len(times) - 1
    p = capi.stb_default_params(alpha, float(times[-1]), n, precision=precision)
    nblk, E = n * (n + 1) // 2, len(tris)
    V = torch.full((nblk, E, E), float("nan"), dtype=torch.float64, device="cuda")
    K = torch.full_like(V, float("nan"))
    ws = torch.empty(capi.stb_assemble_nu_workspace_size(mesh, p, times), dtype=torch.uint8,
                     device="cuda")
    capi.stb_assemble_nu(mesh, p, times, V, K, ws)
    capi.stb_workspace_status(ws)
    return V.cpu().numpy(), K.cpu().numpy()


@pytest.mark.parametrize("name,times,alpha", [
    ("cube2", GRADED, 1.0),
    ("cube4", np.array([0.0, 0.1, 0.15, 0.3, 0.32, 0.5]), 0.6),
    ("ico3", np.array([0.0, 0.25, 0.3, 0.7, 0.75]), 2.0)])
def test_nonuniform_blocks_match_oracle(name, times, alpha):
    nodes, tris = {"cube2": lambda: workloads.cube_mesh(2), "cube4": lambda: workloads.cube_mesh(4),
                   "ico3": lambda: workloads.icosphere(3)}[name]()
    V, K = gpu_assemble_nu(nodes, tris, alpha, times)
    Vo, Ko = oracle.assemble_nu(nodes, tris, alpha, times)
    worst = 0.0
    for b in range(V.shape[0]):
        for got, ref in ((V[b], Vo[b]), (K[b], Ko[b])):
            assert np.all(np.isfinite(got)), b
            rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert rel <= 1e-10, (b, rel)
            worst = max(worst, rel)
    print("%s: non-uniform blocks max rel err %.2e" % (name, worst))


def test_uniform_grid_equals_toeplitz_blocks():
    nodes, tris = workloads.cube_mesh(4)
    n, alpha = 5, 0.9
    times = np.arange(n + 1) * 0.125
    V, K = gpu_assemble_nu(nodes, tris, alpha, times)
    mesh = capi.Mesh(nodes, tris)
    p = capi.stb_default_params(alpha, float(times[-1]), n)
    E = len(tris)
    Vt = torch.empty((n, E, E), dtype=torch.float64, device="cuda")
    Kt = torch.empty_like(Vt)
    ws = torch.empty(capi.stb_assemble_workspace_size(mesh, p), dtype=torch.uint8, device="cuda")
    capi.stb_assemble(mesh, p, Vt, Kt, ws)
    Vt, Kt = Vt.cpu().numpy(), Kt.cpu().numpy()
    for k in range(n):
        for i in range(k + 1):
            b = oracle.block_index(k, i)
            for got, ref in ((V[b], Vt[k - i]), (K[b], Kt[k - i])):
                assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref), (k, i)


def test_matvec_and_solve_match_oracle():
    nodes, tris = workloads.cube_mesh(2)
    Vo, _ = oracle.assemble_nu(nodes, tris, 1.0, GRADED)
    n, E = len(GRADED) - 1, len(tris)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(3, n, E))
    Vd = torch.tensor(Vo, device="cuda")
    y = torch.empty((3, n, E), dtype=torch.float64, device="cuda")
    capi.stb_matvec_nu(Vd, E, n, 3, torch.tensor(x, device="cuda"), y)
    yo = oracle.matvec_nu(Vo, x)
    assert np.abs(y.cpu().numpy() - yo).max() <= 1e-13 * np.abs(yo).max()
    f = rng.normal(size=(3, n, E))
    w = torch.empty_like(y)
    ws = torch.empty(capi.stb_solve_nu_workspace_size(E, n, 3), dtype=torch.uint8, device="cuda")
    capi.stb_solve_nu(Vd, E, n, 3, torch.tensor(f, device="cuda"), w, ws)
    wo = oracle.solve_nu(Vo, f)
    assert np.linalg.norm(w.cpu().numpy() - wo) <= 1e-10 * np.linalg.norm(wo)


def test_nonuniform_pipeline_matches_oracle_pipeline():
    """Dirichlet problem on a graded grid (cube, 192 triangles, steps from
    0.02 to 0.25): every GPU step against the oracle's."""
    nodes, tris = workloads.cube_mesh(4)
    alpha = 1.0
    src = workloads.point_source((1.5, 1.5, 1.5), t0=0.0)
    prob = pipeline.NonUniformDirichletProblem(nodes, tris, alpha, GRADED, src)
    prob.run()
    Vo, Ko = oracle.assemble_nu(nodes, tris, alpha, GRADED)
    area, _ = oracle.triangle_geometry(nodes, tris)
    go = oracle.project_dirichlet_nu(nodes, tris, alpha, GRADED, src)
    assert np.abs(prob.g.cpu().numpy() - go).max() <= 1e-13 * np.abs(go).max()
    fo = oracle.dirichlet_rhs_nu(area, Ko, GRADED, go)
    wo = oracle.solve_nu(Vo, fo)
    w = prob.w.cpu().numpy()
    assert np.linalg.norm(w - wo) / np.linalg.norm(wo) < 1e-8
    e2, r2 = oracle.neumann_error_nu(nodes, tris, alpha, GRADED, src, wo)
    assert abs(prob.relative_error() - math.sqrt(e2 / r2)) < 1e-8
    print("graded grid: L2 error of w_h %.4f" % prob.relative_error())


# ---- mixed precision -------------------------------------------------------------
# Separated pairs in FP32 (closed forms over the corner differences where the
# gap is below the shorter interval, Gauss nodes on the overlap trapezoid
# elsewhere), touching pairs in FP64, blocks stored FP64.  The stated bound
# of the uniform mixed path: relative Frobenius error per block <= 2e-6
# against the FP64 oracle.
MIXED_BOUND = 2e-6


def geometric(n, ratio, T=1.0):
    steps = ratio ** np.arange(n)
    t = np.concatenate([[0.0], np.cumsum(steps / steps.sum())]) * T
    t[-1] = T
    return t


# graded steps; a grid whose small steps sit between long ones (gaps below
# the shorter interval away from k = i + 1, long plateaus cut geometrically);
# a geometric grid; a uniform grid (shared evaluations); small and large alpha
@pytest.mark.parametrize("name,times,alpha", [
    ("cube2", GRADED, 1.0),
    ("cube2", np.array([0.0, 0.3, 0.31, 0.32, 0.7, 0.705, 1.4]), 0.4),
    ("cube4", geometric(10, 1.2), 0.5),
    ("cube4", np.arange(9) / 8.0, 1.0),
    ("ico2", np.array([0.0, 0.01, 0.2, 0.21, 0.5]), 5.0),
    ("cube2", geometric(24, 1.1, 2.0), 0.1)])
def test_nonuniform_mixed_blocks_match_oracle(name, times, alpha):
    nodes, tris = {"cube2": lambda: workloads.cube_mesh(2), "cube4": lambda: workloads.cube_mesh(4),
                   "ico2": lambda: workloads.icosphere(2)}[name]()
    V, K = gpu_assemble_nu(nodes, tris, alpha, times, precision=capi.STB_PREC_MIXED)
    Vo, Ko = oracle.assemble_nu(nodes, tris, alpha, times)
    worst = [0.0, 0.0]
    for b in range(V.shape[0]):
        for c, (got, ref) in enumerate(((V[b], Vo[b]), (K[b], Ko[b]))):
            assert np.all(np.isfinite(got)), b
            rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert rel <= MIXED_BOUND, (b, "VK"[c], rel)
            worst[c] = max(worst[c], rel)
    print("%s, %d steps: mixed non-uniform max block error V %.2e K %.2e"
          % (name, len(times) - 1, worst[0], worst[1]))


def test_nonuniform_mixed_pipeline():
    """The mixed assembly inside the Dirichlet pipeline: the solution within
    a small multiple of the stated block bound of the FP64 pipeline's."""
    nodes, tris = workloads.cube_mesh(4)
    src = workloads.point_source((1.5, 1.5, 1.5), t0=0.0)
    times = geometric(12, 1.2)
    ref = pipeline.NonUniformDirichletProblem(nodes, tris, 1.0, times, src)
    ref.run()
    mix = pipeline.NonUniformDirichletProblem(nodes, tris, 1.0, times, src,
                                              precision=capi.STB_PREC_MIXED)
    mix.run()
    w0, w1 = ref.w.cpu().numpy(), mix.w.cpu().numpy()
    assert np.linalg.norm(w1 - w0) / np.linalg.norm(w0) < 1e-4
    assert abs(mix.relative_error() - ref.relative_error()) < 1e-4


# edge cases of the mixed path: one and two steps (closed forms only, and
# the hat-plus-remainder form of unequal neighbouring steps), the
# icosahedron (20 triangles, half the ordered pairs touching) and its
# 80-triangle refinement (trial-triangle counts below one CTA)
@pytest.mark.parametrize("name,times,alpha", [
    ("cube2", np.array([0.0, 0.4]), 1.0),
    ("cube2", np.array([0.0, 0.1, 0.5]), 0.7),
    ("ico20", np.array([0.0, 0.2, 0.25, 0.6]), 1.5),
    ("ico80", np.array([0.0, 0.05, 0.3, 0.31, 0.9]), 0.3)])
def test_nonuniform_mixed_edge_cases(name, times, alpha):
    nodes, tris = {"cube2": lambda: workloads.cube_mesh(2), "ico20": lambda: workloads.icosphere(1),
                   "ico80": lambda: workloads.icosphere(2)}[name]()
    V, K = gpu_assemble_nu(nodes, tris, alpha, times, precision=capi.STB_PREC_MIXED)
    Vo, Ko = oracle.assemble_nu(nodes, tris, alpha, times)
    for b in range(V.shape[0]):
        for c, (got, ref) in enumerate(((V[b], Vo[b]), (K[b], Ko[b]))):
            assert np.all(np.isfinite(got)), b
            nr = np.linalg.norm(ref)
            if nr == 0.0:  # K of a flat closed surface's identical pairs only
                assert np.linalg.norm(got) <= 1e-12, (b, "VK"[c])
                continue
            rel = np.linalg.norm(got - ref) / nr
            assert rel <= MIXED_BOUND, (b, "VK"[c], rel)
