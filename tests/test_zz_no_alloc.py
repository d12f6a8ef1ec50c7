"""The allocation-free block-Toeplitz product (stb_toeplitz_matvec_static).

Some callers cannot allocate device memory where they call the library: a
stream being captured into a CUDA graph, a plugin whose host framework owns
all device memory, real-time code that allocates only at start-up.  For them
the library keeps the product's partial sums in a fixed scratch array of its
own.  This test calls that entry point through the C ABI and checks it against
the workspace version on two calls in a row and on a larger problem followed
by a smaller one, with FP64 and FP32 blocks (the scratch keeps the previous
call's contents, which must not leak into the next result), and that a
problem larger than the scratch is refused.  It lives in its own file, named
so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2102_09811_gb300 import capi

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


def _compare(A, storage, E, n_steps, nrhs, rng, beta=0.25):
    """One call of each entry point with the same x and y0: results equal to
    rounding (the same kernels, only the scratch differs)."""
    ws = torch.empty(capi.stb_toeplitz_workspace_size(E, n_steps, nrhs), dtype=torch.uint8,
                     device="cuda")
    x = torch.tensor(rng.normal(size=(nrhs, n_steps, E)), device="cuda")
    y0 = torch.tensor(rng.normal(size=(nrhs, n_steps, E)), device="cuda")
    y_ref = y0.clone()
    y_new = y0.clone()
    capi.stb_toeplitz_matvec(A, storage, E, n_steps, nrhs, x, beta, y_ref, ws)
    capi.stb_toeplitz_matvec_static(A, storage, E, n_steps, nrhs, x, beta, y_new)
    torch.cuda.synchronize()
    scale = float(A.abs().max()) * E * n_steps * float(x.abs().max())
    return float((y_new - y_ref).abs().max()), scale


@pytest.mark.parametrize("storage", [capi.STB_STORE_F64, capi.STB_STORE_F32])
def test_static_scratch_matvec_matches_workspace_matvec(storage):
    """Two calls in a row of one shape, then a larger problem (more partial
    slices in the scratch) followed by a smaller one: slices left behind by
    an earlier, larger call must not reach a later result."""
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    torch.cuda.set_device(0)
    rng = np.random.default_rng(23)
    dt = torch.float64 if storage == capi.STB_STORE_F64 else torch.float32
    for E, n_steps, nrhs in ((300, 13, 2), (300, 13, 2), (400, 40, 3), (250, 9, 1)):
        A = torch.tensor(rng.normal(size=(n_steps, E, E)), device="cuda", dtype=dt)
        diff, scale = _compare(A, storage, E, n_steps, nrhs, rng)
        assert diff <= 4 * EPS * scale, (E, n_steps, nrhs, diff)


def test_static_scratch_rejects_oversized_problems():
    lib = capi._library()
    E, n_steps, nrhs = 3072, 64, 8  # needs 8 * 8 * 64 * 3072 * 8 bytes > 16 MiB
    A = torch.empty(1, dtype=torch.float64, device="cuda")
    x = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = lib.stb_toeplitz_matvec_static(ctypes.c_void_p(A.data_ptr()), capi.STB_STORE_F64, E,
                                        n_steps, nrhs, ctypes.c_void_p(x.data_ptr()), 0.0,
                                        ctypes.c_void_p(x.data_ptr()), None)
    assert rc == -1
    assert "static scratch" in lib.stb_last_error_message().decode()
