"""CPU checks of the C ABI: the library loads, exports every function that
include/stbem.h declares, and its host-side argument and mesh validation
answers with the documented status codes (no GPU work is started)."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads
from paper_2102_09811_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "stbem.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stb_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    lib = ctypes.CDLL(capi.library_path())
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_function():
    assert set(declared_functions()) <= set(capi._SIGS)


def test_status_strings_and_defaults():
    lib = capi._library()
    for code in range(-8, 1):
        assert lib.stb_status_string(code).decode() not in ("", "unknown status")
    p = capi.stb_default_params(0.5, 2.0, 10)
    assert (p.alpha, p.T, p.n_steps, p.quad_regular, p.quad_singular, p.precision, p.storage,
            p.flags) == (0.5, 2.0, 10, 3, 4, 0, 0, 0)


def test_launch_count_starts_without_gpu_work():
    assert capi.stb_launch_count() >= 0


def _create(nodes, tris):
    lib = capi._library()
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    h = ctypes.c_void_p()
    rc = lib.stb_mesh_create(nodes.ctypes.data_as(ctypes.c_void_p), nodes.shape[0],
                             tris.ctypes.data_as(ctypes.c_void_p), tris.shape[0], ctypes.byref(h))
    return rc, lib.stb_last_error_message().decode()


def test_mesh_validation_rejects_bad_surfaces():
    nodes, tris = workloads.cube_mesh(1)
    rc, msg = _create(nodes, tris[:-1])  # one triangle missing: not closed
    assert rc == -2 and "opposite" in msg
    flipped = tris.copy()
    flipped[0] = flipped[0][[0, 2, 1]]  # inconsistent orientation
    assert _create(nodes, flipped)[0] == -2
    bad = tris.copy()
    bad[3, 1] = bad[3, 0]  # repeated vertex
    assert _create(nodes, bad)[0] == -2
    bad = tris.copy()
    bad[2, 2] = 999  # index out of range
    assert _create(nodes, bad)[0] == -2
    nn = nodes.copy()
    nn[0, 0] = np.nan
    assert _create(nn, tris)[0] == -2
    assert _create(nodes, tris[:3])[0] == -1  # too few triangles


def test_null_arguments():
    lib = capi._library()
    n = ctypes.c_size_t()
    assert lib.stb_assemble_workspace_size(None, None, ctypes.byref(n)) == -1
    assert lib.stb_toeplitz_workspace_size(0, 1, 1, ctypes.byref(n)) == -1
    assert lib.stb_toeplitz_workspace_size(10, 4, 2, ctypes.byref(n)) == 0 and n.value > 256
