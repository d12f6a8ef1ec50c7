"""Full-size parity of the sphere workloads (icosphere, 5120 triangles, radius
1): mixed assembly checked on sampled rows against the FP64 oracle, the
refined mixed solve checked by an independent FP64 residual on the GPU, and
the tensor-core product against the FP64 product.

  sphere5120_e128: 128 steps, alpha = 1, one exterior source;
  sphere5120_e256: 256 steps, alpha = 1, eight exterior sources solved as
                   eight right-hand sides, blocks stored in FP32 (26.8 GB per
                   matrix).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2102_09811_gb300 import capi, pipeline

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
MIXED_BOUND = 2e-6  # stated per-block relative Frobenius bound of the mixed assembly


@pytest.fixture(scope="module", autouse=True)
def cuda_device():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)


def _run_mixed(name):
    wl = workloads.workload(name)
    prob = pipeline.DirichletProblem(wl["nodes"], wl["tris"], wl["alpha"], wl["T"], wl["n_steps"],
                                     wl["sources"], precision=capi.STB_PREC_MIXED,
                                     storage=capi.STB_STORE_F32)
    prob.run()
    torch.cuda.synchronize()
    return wl, prob


def _check_rows(wl, prob, rows):
    """Mixed blocks on sampled rows (every block d) against the FP64 oracle."""
    n = wl["n_steps"]
    Vo, Ko = oracle.assemble_rows(wl["nodes"], wl["tris"], wl["alpha"], wl["T"], n, rows)
    idx = torch.tensor(rows, device="cuda")
    Vg = prob.V.index_select(1, idx).double().cpu().numpy().transpose(1, 0, 2)
    Kg = prob.K.index_select(1, idx).double().cpu().numpy().transpose(1, 0, 2)
    ev = [np.linalg.norm(Vg[:, d] - Vo[:, d]) / np.linalg.norm(Vo[:, d]) for d in range(n)]
    ek = [np.linalg.norm(Kg[:, d] - Ko[:, d]) / np.linalg.norm(Ko[:, d]) for d in range(n)]
    assert max(ev) < MIXED_BOUND and max(ek) < MIXED_BOUND, (max(ev), max(ek))
    return max(ev), max(ek)


def _fp64_residual(prob):
    """||f - V_h w|| / ||f|| with the FP64-arithmetic product (not the
    double-float product that the refinement itself uses)."""
    E, n, nrhs = prob.E, prob.n_steps, prob.nrhs
    ws = torch.empty(capi.stb_toeplitz_workspace_size(E, n, nrhs), dtype=torch.uint8, device="cuda")
    y = torch.empty_like(prob.w)
    capi.stb_toeplitz_matvec(prob.V, capi.STB_STORE_F32, E, n, nrhs, prob.w, 0.0, y, ws)
    torch.cuda.synchronize()
    return float(torch.linalg.norm(prob.f - y) / torch.linalg.norm(prob.f))


def test_sphere5120_e128_mixed():
    wl, prob = _run_mixed("sphere5120_e128")
    ev, ek = _check_rows(wl, prob, np.array([0, 2560, 5119]))
    it, rep = capi.stb_solve_report(prob.ws_solve)
    assert 1 <= it <= 8 and rep <= 1e-10, (it, rep)
    res = _fp64_residual(prob)
    assert res <= 2e-10, res
    rel = prob.relative_error()
    assert np.isfinite(rel) and rel < 0.5, rel
    # tensor-core product of the assembled V against the FP64 product
    E, n = prob.E, prob.n_steps
    y64 = torch.empty_like(prob.w)
    ytc = torch.empty_like(prob.w)
    for arith, y in ((capi.STB_ARITH_FP64, y64), (capi.STB_ARITH_TF32, ytc)):
        ws = torch.empty(capi.stb_toeplitz_ex_workspace_size(E, n, 1, arith), dtype=torch.uint8,
                         device="cuda")
        capi.stb_toeplitz_matvec_ex(prob.V, capi.STB_STORE_F32, E, n, 1, prob.w, 0.0, y, arith, ws)
        capi.stb_workspace_status(ws)
    rel_tc = float(torch.linalg.norm(ytc - y64) / torch.linalg.norm(y64))
    assert rel_tc < 2e-3, rel_tc
    print("sphere5120_e128: block error V %.2e K %.2e; %d refinements, residual %.2e (FP64 %.2e); "
          "L2 error %.4f; TF32 product rel %.2e" % (ev, ek, it, rep, res, rel, rel_tc))


def test_sphere5120_e256_eight_sources():
    wl, prob = _run_mixed("sphere5120_e256")
    assert prob.nrhs == 8
    ev, ek = _check_rows(wl, prob, np.array([17, 4000]))
    it, rep = capi.stb_solve_report(prob.ws_solve)
    assert 1 <= it <= 8 and rep <= 1e-10, (it, rep)
    res = _fp64_residual(prob)
    assert res <= 2e-10, res
    rel = prob.relative_error()
    assert np.isfinite(rel) and rel < 0.5, rel
    print("sphere5120_e256 (8 rhs): block error V %.2e K %.2e; %d refinements, residual %.2e "
          "(FP64 %.2e); L2 error %.4f" % (ev, ek, it, rep, res, rel))
