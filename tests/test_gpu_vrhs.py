"""The matrix-free right-hand side: V and f = (1/2 M_h + K_h) g with K's
blocks contracted as they are formed, never stored (the fused K g of the
scope table's last row).  V must equal the stored-path V bit for bit (the
same arithmetic); f is compared with the stored path (FP32 K times g in
double-float arithmetic) and with the FP64 oracle's (1/2 M + K) g within
the mixed block bound (2e-6, relative 2-norm per step)."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2102_09811_gb300 import capi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_device():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    capi._library()


def _stored_and_fused(nodes, tris, alpha, T, n, g):
    mesh = capi.Mesh(nodes, tris)
    p = capi.stb_default_params(alpha, T, n, precision=capi.STB_PREC_MIXED,
                                storage=capi.STB_STORE_F32)
    E, nrhs = len(tris), g.shape[0]
    gd = torch.tensor(g, device="cuda")
    V = torch.empty((n, E, E), dtype=torch.float32, device="cuda")
    K = torch.empty_like(V)
    ws = torch.empty(capi.stb_assemble_workspace_size(mesh, p), dtype=torch.uint8, device="cuda")
    capi.stb_assemble(mesh, p, V, K, ws)
    f = torch.empty((nrhs, n, E), dtype=torch.float64, device="cuda")
    ws = torch.empty(capi.stb_rhs_workspace_size(mesh, p, nrhs), dtype=torch.uint8, device="cuda")
    capi.stb_dirichlet_rhs(mesh, p, K, gd, nrhs, f, ws)
    Vf = torch.full_like(V, float("nan"))
    ff = torch.full_like(f, float("nan"))
    ws = torch.empty(capi.stb_assemble_vrhs_workspace_size(mesh, p, nrhs), dtype=torch.uint8,
                     device="cuda")
    capi.stb_assemble_vrhs(mesh, p, Vf, gd, nrhs, ff, ws)
    capi.stb_workspace_status(ws)
    return V, f, Vf, ff, K


@pytest.mark.parametrize("name,n,nrhs", [("cube4", 16, 1), ("cube4", 16, 3), ("ico3", 9, 2),
                                         ("cube2", 40, 3), ("cube2", 1, 1)])
def test_vrhs_matches_stored_path_and_oracle(name, n, nrhs):
    nodes, tris = {"cube4": lambda: workloads.cube_mesh(4), "cube2": lambda: workloads.cube_mesh(2),
                   "ico3": lambda: workloads.icosphere(3)}[name]()
    alpha, T = 0.9, 1.0
    rng = np.random.default_rng(n * 10 + nrhs)
    g = rng.normal(size=(nrhs, n, len(tris)))
    V, f, Vf, ff, K = _stored_and_fused(nodes, tris, alpha, T, n, g)
    assert torch.equal(V, Vf)
    f, ff = f.cpu().numpy(), ff.cpu().numpy()
    Vo, Ko = oracle.assemble(nodes, tris, alpha, T, n)
    area, _ = oracle.triangle_geometry(nodes, tris)
    fo = oracle.dirichlet_rhs(area, Ko, g, T)
    worst = 0.0
    for r in range(nrhs):
        for k in range(n):
            nrm = np.linalg.norm(fo[r, k])
            e_std = np.linalg.norm(ff[r, k] - f[r, k]) / nrm
            e_orc = np.linalg.norm(ff[r, k] - fo[r, k]) / nrm
            assert e_std <= 2e-6 and e_orc <= 2e-6, (r, k, e_std, e_orc)
            worst = max(worst, e_orc)
    print("%s n=%d nrhs=%d: matrix-free f vs oracle %.2e" % (name, n, nrhs, worst))


def test_vrhs_bench_workload():
    """3072 triangles, 64 steps, alpha 0.5 (the bench workload): V bit for
    bit, f against the stored path."""
    wl = workloads.workload("cube3072_e64")
    g = np.random.default_rng(64).normal(size=(1, 64, len(wl["tris"])))
    V, f, Vf, ff, K = _stored_and_fused(wl["nodes"], wl["tris"], 0.5, wl["T"], 64, g)
    assert torch.equal(V, Vf)
    rel = (torch.linalg.norm(ff - f, dim=2) / torch.linalg.norm(f, dim=2)).max().item()
    assert rel <= 2e-6, rel
    print("bench workload: matrix-free f vs stored path %.2e" % rel)


def test_vrhs_rejects():
    nodes, tris = workloads.cube_mesh(2)
    mesh = capi.Mesh(nodes, tris)
    p = capi.stb_default_params(1.0, 1.0, 65, precision=capi.STB_PREC_MIXED,
                                storage=capi.STB_STORE_F32)
    with pytest.raises(capi.StbError):
        capi.stb_assemble_vrhs_workspace_size(mesh, p, 2)  # 2 x 65 > 128
    p = capi.stb_default_params(1.0, 1.0, 4)
    with pytest.raises(capi.StbError):
        capi.stb_assemble_vrhs_workspace_size(mesh, p, 1)  # FP64
