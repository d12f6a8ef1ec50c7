"""Batched assembly of many independent problems (64 ellipsoids from seed 0:
320..5120 triangles, 16..128 steps, alpha in [0.1, 10]) in memory-budgeted
waves, each wave one persistent launch for all pair classes (the touching
pairs first, then the separated pairs).

Checks: the batch writes the same blocks as the single-problem assembly
(bit for bit, either tile), the tile autotuner returns a valid tile, and the
blocks match the FP64 oracle per block within the stated mixed bound: every
row of the four smallest meshes, one seeded row of every other mesh (64
rows), the oracle run on host threads.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2102_09811_gb300 import capi

pytestmark = pytest.mark.gpu
MIXED_BOUND = 2e-6
WAVE_BYTES = 40e9  # V + K of one wave


@pytest.fixture(scope="module", autouse=True)
def cuda_device():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)


def _params(p):
    return capi.stb_default_params(p["alpha"], p["T"], p["n_steps"], precision=capi.STB_PREC_MIXED,
                                   storage=capi.STB_STORE_F32)


def _alloc(p, with_k=True):
    E, n = len(p["tris"]), p["n_steps"]
    V = torch.empty((n, E, E), dtype=torch.float32, device="cuda")
    K = torch.empty((n, E, E), dtype=torch.float32, device="cuda") if with_k else None
    return V, K


def _batch(probs, meshes, tile, with_k=True):
    VK = [_alloc(p, with_k) for p in probs]
    V, K = [v for v, _ in VK], [k for _, k in VK]
    params = [_params(p) for p in probs]
    ws = torch.empty(capi.stb_batch_workspace_size(meshes, params, V, K), dtype=torch.uint8,
                     device="cuda")
    capi.stb_batch_assemble(meshes, params, V, K, tile, ws)
    capi.stb_workspace_status(ws)
    return V, K


def _single(p, mesh):
    V, K = _alloc(p)
    prm = _params(p)
    ws = torch.empty(capi.stb_assemble_workspace_size(mesh, prm), dtype=torch.uint8, device="cuda")
    capi.stb_assemble(mesh, prm, V, K, ws)
    capi.stb_workspace_status(ws)
    return V, K


def test_batch_equals_single_problem_assembly_for_every_tile():
    """Both tiles write the single-problem blocks bit for bit (the touching
    pairs run on 128 threads of the CTA whatever its size)."""
    probs = workloads.batch_workload(seed=0)[:6]
    meshes = [capi.Mesh(p["nodes"], p["tris"]) for p in probs]
    ref = [_single(p, m) for p, m in zip(probs, meshes)]
    for tile in (128, 256):
        V, K = _batch(probs, meshes, tile)
        for i in range(len(probs)):
            assert torch.equal(V[i], ref[i][0]), (tile, i)
            assert torch.equal(K[i], ref[i][1]), (tile, i)
    # V only
    V, K = _batch(probs[:2], meshes[:2], 128, with_k=False)
    assert torch.equal(V[0], ref[0][0]) and torch.equal(V[1], ref[1][0])


def test_batch_tuner_picks_a_tile():
    probs = workloads.batch_workload(seed=0)[:8]
    meshes = [capi.Mesh(p["nodes"], p["tris"]) for p in probs]
    VK = [_alloc(p) for p in probs]
    V, K = [v for v, _ in VK], [k for _, k in VK]
    params = [_params(p) for p in probs]
    ws = torch.empty(capi.stb_batch_workspace_size(meshes, params, V, K), dtype=torch.uint8,
                     device="cuda")
    tile = capi.stb_batch_tune(meshes, params, V, K, ws)
    assert tile in (128, 256)
    capi.stb_batch_assemble(meshes, params, V, K, 0, ws)  # the tuned tile
    capi.stb_workspace_status(ws)
    print("tuned tile: %d columns per work item" % tile)


def _waves(probs):
    order = sorted(range(len(probs)), key=lambda i: -len(probs[i]["tris"]) ** 2 * probs[i]["n_steps"])
    waves, cur, size = [], [], 0.0
    for i in order:
        b = 8.0 * len(probs[i]["tris"]) ** 2 * probs[i]["n_steps"]
        if cur and size + b > WAVE_BYTES:
            waves.append(cur)
            cur, size = [], 0.0
        cur.append(i)
        size += b
    waves.append(cur)
    return waves


@pytest.mark.slow
def test_batch_of_64_ellipsoids_against_oracle():
    probs = workloads.batch_workload(seed=0)
    assert len(probs) == 64
    rng = np.random.default_rng(64)
    sizes = np.array([len(p["tris"]) for p in probs])
    smallest = set(np.argsort(sizes, kind="stable")[:4].tolist())
    rows = {i: (np.arange(sizes[i]) if i in smallest else rng.integers(0, sizes[i], size=1))
            for i in range(64)}
    worst = [0.0, 0.0]
    pool = ThreadPoolExecutor(max_workers=16)
    for wave in _waves(probs):
        wp = [probs[i] for i in wave]
        meshes = [capi.Mesh(p["nodes"], p["tris"]) for p in wp]
        V, K = _batch(wp, meshes, 0)
        jobs = [pool.submit(oracle.assemble_rows, p["nodes"], p["tris"], p["alpha"], p["T"],
                            p["n_steps"], rows[i]) for i, p in zip(wave, wp)]
        for k, (i, p) in enumerate(zip(wave, wp)):
            Vo, Ko = jobs[k].result()
            idx = torch.tensor(rows[i], device="cuda")
            Vg = V[k].index_select(1, idx).double().cpu().numpy().transpose(1, 0, 2)
            Kg = K[k].index_select(1, idx).double().cpu().numpy().transpose(1, 0, 2)
            for d in range(p["n_steps"]):
                ev = np.linalg.norm(Vg[:, d] - Vo[:, d]) / np.linalg.norm(Vo[:, d])
                ek = np.linalg.norm(Kg[:, d] - Ko[:, d]) / np.linalg.norm(Ko[:, d])
                assert ev < MIXED_BOUND and ek < MIXED_BOUND, (i, d, ev, ek)
                worst = [max(worst[0], ev), max(worst[1], ek)]
        del V, K
        torch.cuda.empty_cache()
    pool.shutdown()
    print("64-ellipsoid batch: max block error V %.2e K %.2e" % tuple(worst))


def test_graph_captured_batch_pipeline():
    """Assembly, projection, right-hand side, solve and error of six problems
    in three waves, each wave one CUDA graph: replays reproduce the first run
    exactly, every captured solve reaches the 1e-10 residual with the
    refinement count of the synchronous first pass, and the solutions equal
    those of the one-problem pipeline."""
    from paper_2102_09811_gb300 import pipeline
    probs = workloads.batch_workload(seed=0)[:6]
    bp = pipeline.BatchPipeline(probs, wave_bytes=16e9)
    assert len(bp.waves) == 3
    bp.run()
    torch.cuda.synchronize()
    first = [it["w"].clone() for it in bp.items]
    errs = bp.relative_errors()
    bp.run()  # graph replays
    torch.cuda.synchronize()
    for a, it in zip(first, bp.items):
        assert torch.equal(a, it["w"])
    for r, res, st in bp.reports():
        assert st == 0 and 1 <= r <= 8 and res <= 1e-10, (r, res, st)
    for k, p in enumerate(probs):
        dp = pipeline.DirichletProblem(p["nodes"], p["tris"], p["alpha"], p["T"], p["n_steps"],
                                       p["sources"], precision=capi.STB_PREC_MIXED,
                                       storage=capi.STB_STORE_F32)
        dp.run()
        rel = float(torch.linalg.norm(dp.w - bp.items[k]["w"]) / torch.linalg.norm(dp.w))
        assert rel <= 1e-12, (k, rel)
        assert abs(dp.relative_error() - errs[k]) <= 1e-12 * errs[k], (k, dp.relative_error(), errs[k])
        del dp
        torch.cuda.empty_cache()
    print("graph-captured batch: 6 problems in 3 waves, L2 errors",
          " ".join("%.4f" % e for e in errs))
