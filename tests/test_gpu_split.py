"""GPU: the split-operand block-Toeplitz product on the tensor cores
(STB_ARITH_SPLIT, eq. V_mat) against the FP64 oracle product of the same FP32
blocks, and the expiry paths of the bounded device waits (mbarrier waits of
the tensor-core kernels, grid barriers of the cooperative kernels).

Bounds.  Per row, block and chunk of 64 columns, and per step vector and
chunk of x, the split product scales by 2^-e (2^-g), 2^e the power of two
just above the chunk's largest magnitude, and keeps five 9-bit digit slices
(44 bits); the products of levels 0..3 are exact in FP32.  In units of
2^(e+g) its error per chunk is at most 64 x 6.1 x 2^-45 = 2^-36.4 from the
dropped digits and levels plus 2^-34.4 from one rounding of the chunk's low
part: below 2^-33.  The tests require that rigorous bound everywhere and,
on data whose chunks are not dominated by single entries (Gaussian), the
bound of the double-float product, 2^-40 sum_d |A^d| |x^{k-d}| entrywise;
on assembled V and K blocks they require 2^-40 in norm.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2102_09811_gb300 import capi, pipeline

pytestmark = pytest.mark.gpu
CH = 64


@pytest.fixture(scope="module", autouse=True)
def cuda_device():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    capi._library()


def split_matvec(A32, x, y0, beta, arith=capi.STB_ARITH_SPLIT):
    n_steps, E = A32.shape[0], A32.shape[1]
    nrhs = x.shape[0]
    Ad = torch.tensor(A32, dtype=torch.float32, device="cuda")
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.tensor(y0, dtype=torch.float64, device="cuda")
    ws = torch.empty(capi.stb_toeplitz_ex_workspace_size(E, n_steps, nrhs, arith), dtype=torch.uint8,
                     device="cuda")
    capi.stb_toeplitz_matvec_ex(Ad, capi.STB_STORE_F32, E, n_steps, nrhs, xd, beta, yd, arith, ws)
    capi.stb_workspace_status(ws)
    return yd.cpu().numpy()


def pow2_above(m):
    """Smallest power of two strictly above m (0 where m == 0)."""
    out = np.zeros_like(m)
    nz = m > 0
    out[nz] = np.exp2(np.floor(np.log2(m[nz])) + 1.0)
    return out


def chunk_bound(A, x):
    """2^-33 sum_{d <= k} sum_chunks 2^(e+g): [nrhs, n_steps, E]."""
    n_steps, E, _ = A.shape
    nrhs = x.shape[0]
    nc = (E + CH - 1) // CH
    pad = nc * CH - E
    Ap = np.pad(np.abs(A), ((0, 0), (0, 0), (0, pad))).reshape(n_steps, E, nc, CH).max(axis=3)
    xp = np.pad(np.abs(x), ((0, 0), (0, 0), (0, pad))).reshape(nrhs, n_steps, nc, CH).max(axis=3)
    eA, gX = pow2_above(Ap), pow2_above(xp)
    b = np.zeros((nrhs, n_steps, E))
    for d in range(n_steps):
        # rows l, vectors m: sum over chunks of eA[d, l, c] gX[r, m, c]
        t = np.einsum("lc,rmc->rml", eA[d], gX[:, : n_steps - d])
        b[:, d:] += t
    return 2.0 ** -33 * b


def check(A, x, y0, beta, entrywise_40=True):
    got = split_matvec(A, x, y0, beta)
    exact = beta * y0 + oracle.toeplitz_matvec(A, x)
    mag = oracle.toeplitz_matvec(np.abs(A), np.abs(x)) + abs(beta) * np.abs(y0)
    err = np.abs(got - exact)
    assert np.all(np.isfinite(got))
    cb = chunk_bound(A, x) + 2.0 ** -50 * mag
    assert np.all(err <= cb), float((err / np.where(cb > 0, cb, 1)).max())
    if entrywise_40:
        assert np.all(err <= 2.0 ** -40 * mag), float(np.log2((err / np.where(mag > 0, mag, 1)).max()))
    return err, mag, exact


def test_split_matvec_gaussian():
    """The double-float product's test data and bound."""
    rng = np.random.default_rng(12)
    E, n_steps, nrhs = 150, 13, 2
    A = rng.normal(size=(n_steps, E, E)).astype(np.float32).astype(np.float64)
    x = rng.normal(size=(nrhs, n_steps, E))
    y0 = rng.normal(size=(nrhs, n_steps, E))
    err, mag, _ = check(A, x, y0, 2.0)
    print("split matvec, Gaussian: worst err/(|A||x|) = 2^%.1f" % np.log2((err / mag).max()))


# (E, n_steps, nrhs): one box; two boxes of 64 steps; 3 right-hand sides (4 per
# box, one unused); 5 (8 per box); E not a multiple of 4 (scalar loads) and
# not of 64 / 128; 8 right-hand sides as in the 8-source workload; a single
# triangle; 70 right-hand sides (two groups); one step
@pytest.mark.parametrize("E,n_steps,nrhs", [(256, 16, 1), (200, 70, 1), (200, 11, 3), (132, 9, 5),
                                            (388, 130, 2), (131, 21, 8), (1, 3, 1), (96, 5, 70),
                                            (130, 1, 1)])
def test_split_matvec_shapes(E, n_steps, nrhs):
    rng = np.random.default_rng(E * 1000 + n_steps * 10 + nrhs)
    A = rng.normal(size=(n_steps, E, E)).astype(np.float32).astype(np.float64)
    x = rng.normal(size=(nrhs, n_steps, E))
    y0 = rng.normal(size=(nrhs, n_steps, E))
    check(A, x, y0, -0.75)
    check(A, x, y0, 0.0)


def test_split_matvec_scales_and_zeros():
    """Entries far from 1 (the chunk scales follow them), zero chunks of A and
    zero steps of x, and entries spread over 2^-40 .. 1 inside chunks (only the
    rigorous chunk bound applies there)."""
    rng = np.random.default_rng(5)
    E, n_steps, nrhs = 200, 12, 2
    A = rng.normal(size=(n_steps, E, E)) * 1e-20
    A[:, :, 64:128] = 0.0            # a zero chunk in every row
    A[3] = 0.0                       # a zero block
    x = rng.normal(size=(nrhs, n_steps, E)) * 1e12
    x[:, 5] = 0.0                    # a zero step
    A = A.astype(np.float32).astype(np.float64)
    check(A, x, np.zeros_like(x), 0.0)
    A2 = (rng.normal(size=(n_steps, E, E)) * np.exp2(rng.uniform(-40, 0, size=(n_steps, E, E))))
    A2 = A2.astype(np.float32).astype(np.float64)
    x2 = rng.normal(size=(nrhs, n_steps, E)) * np.exp2(rng.uniform(-30, 0, size=(nrhs, n_steps, E)))
    err, mag, exact = check(A2, x2, np.zeros_like(x2), 0.0, entrywise_40=False)
    # random signs cancel in y while the error follows the chunk scales
    rel = np.linalg.norm(err) / np.linalg.norm(exact)
    assert rel <= 2.0 ** -38, rel


@pytest.fixture(scope="module")
def c1_mixed():
    wl = workloads.workload("cube192_e16")
    nodes, tris, alpha, T, n, src = (wl["nodes"], wl["tris"], wl["alpha"], wl["T"], wl["n_steps"],
                                     wl["sources"])
    prob = pipeline.DirichletProblem(nodes, tris, alpha, T, n, src, precision=capi.STB_PREC_MIXED,
                                     storage=capi.STB_STORE_F32)
    prob.run()
    torch.cuda.synchronize()
    return (prob.V.double().cpu().numpy(), prob.K.double().cpu().numpy(), prob.g.cpu().numpy(),
            prob.w.cpu().numpy())


def test_split_matvec_assembled_blocks(c1_mixed):
    """V w and K g with the assembled FP32 blocks of the 192-triangle cube:
    the chunk bound entrywise, 2^-40 in norm (single-block steps concentrate
    the rows' magnitude in a few near-field entries, so the entrywise
    2^-40 |A||x| bound is not claimed)."""
    V, K, g, w = c1_mixed
    for A, x in ((V, w), (K, g)):
        err, mag, exact = check(A, x, np.zeros_like(x), 0.0, entrywise_40=False)
        rel = np.linalg.norm(err) / np.linalg.norm(exact)
        assert rel <= 2.0 ** -40, rel
        print("split matvec, assembled blocks: normwise 2^%.1f" % np.log2(rel))


def test_bounded_wait_expires_without_fault():
    """A device wait on a barrier that nothing arrives on expires after its
    limit: the status word reads STB_ERR_TIMEOUT, the context stays usable."""
    probe = torch.arange(64, dtype=torch.float32, device="cuda")  # 256 bytes
    ws = torch.empty(256, dtype=torch.uint8, device="cuda")
    capi.stb_selftest_bounded_wait(probe, 1_000_000, arrive=True, workspace=ws)
    capi.stb_workspace_status(ws)  # completes: STB_OK
    capi.stb_selftest_bounded_wait(probe, 1_000_000, arrive=False, workspace=ws)
    with pytest.raises(capi.StbError) as e:
        capi.stb_workspace_status(ws)
    assert e.value.code == -7
    assert "expired" in str(e.value).lower()
    # the context still works
    rng = np.random.default_rng(1)
    A = rng.normal(size=(3, 64, 64)).astype(np.float32).astype(np.float64)
    x = rng.normal(size=(1, 3, 64))
    check(A, x, np.zeros_like(x), 0.0)
    with pytest.raises(capi.StbError):
        capi.stb_selftest_bounded_wait(probe, 10, arrive=False, workspace=ws)


def test_grid_barrier_expires_without_fault():
    """The grid barrier of the cooperative kernels: with every CTA arriving it
    passes (status STB_OK, every CTA reports 1); with one CTA skipping it, the
    others' waits expire after their limit (STB_ERR_TIMEOUT, those CTAs report
    0, the skipping one 2) and the context stays usable."""
    n = 8
    ws = torch.zeros(512 + 4 * n, dtype=torch.uint8, device="cuda")
    capi.stb_selftest_grid_barrier(n, -1, 1_000_000, ws)
    capi.stb_workspace_status(ws)
    out = ws[512:].view(torch.int32).cpu().tolist()
    assert out == [1] * n, out
    capi.stb_selftest_grid_barrier(n, 3, 1_000_000, ws)
    with pytest.raises(capi.StbError) as e:
        capi.stb_workspace_status(ws)
    assert e.value.code == -7
    out = ws[512:].view(torch.int32).cpu().tolist()
    assert out[3] == 2 and all(v == 0 for i, v in enumerate(out) if i != 3), out
    with pytest.raises(capi.StbError):
        capi.stb_selftest_grid_barrier(n, n, 1_000_000, ws)  # skip out of range
    rng = np.random.default_rng(2)
    A = rng.normal(size=(3, 64, 64)).astype(np.float32).astype(np.float64)
    x = rng.normal(size=(1, 3, 64))
    check(A, x, np.zeros_like(x), 0.0)
