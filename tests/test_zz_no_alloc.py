"""The allocation-free block-Toeplitz product (stb_toeplitz_matvec_static).

Some callers cannot allocate device memory where they call the library: a
stream being captured into a CUDA graph, a plugin whose host framework owns
all device memory, real-time code that allocates only at start-up.  For them
the library keeps the product's partial sums in a fixed scratch array of its
own.  This test calls that entry point through the C ABI and checks it against
the workspace version on two calls in a row (the scratch keeps the previous
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


def test_static_scratch_matvec_matches_workspace_matvec():
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    torch.cuda.set_device(0)
    rng = np.random.default_rng(23)
    E, n_steps, nrhs = 300, 13, 2
    A = torch.tensor(rng.normal(size=(n_steps, E, E)), device="cuda")
    ws = torch.empty(capi.stb_toeplitz_workspace_size(E, n_steps, nrhs), dtype=torch.uint8,
                     device="cuda")
    scale = float(A.abs().max()) * E * n_steps
    for call in range(2):
        x = torch.tensor(rng.normal(size=(nrhs, n_steps, E)), device="cuda")
        y0 = torch.tensor(rng.normal(size=(nrhs, n_steps, E)), device="cuda")
        y_ref = y0.clone()
        y_new = y0.clone()
        capi.stb_toeplitz_matvec(A, capi.STB_STORE_F64, E, n_steps, nrhs, x, 0.25, y_ref, ws)
        capi.stb_toeplitz_matvec_static(A, capi.STB_STORE_F64, E, n_steps, nrhs, x, 0.25, y_new)
        torch.cuda.synchronize()
        diff = float((y_new - y_ref).abs().max())
        assert diff <= 4 * EPS * scale * float(x.abs().max()), (call, diff)


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
