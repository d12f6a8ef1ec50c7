"""Thin ctypes binding of the C ABI in include/stbem.h.

Functions carry the C names and only marshal arguments: device buffers are
torch CUDA tensors (their data_ptr is passed), host arrays are numpy arrays,
streams are torch.cuda.Stream objects (or None for the current stream).
Every computation runs in the CUDA library; if the compiled library is missing
this module raises instead of falling back to anything else.
"""
import ctypes
import os

import numpy as np

from . import _build

STB_OK = 0
STB_PREC_FP64, STB_PREC_MIXED = 0, 1
STB_STORE_F64, STB_STORE_F32 = 0, 1
STB_ARITH_FP64, STB_ARITH_DF, STB_ARITH_TF32, STB_ARITH_SPLIT = 0, 1, 2, 3
STB_FLAG_NO_SYNC = 1


def STB_FLAG_REFINE(n):
    return (n & 15) << 8



_lib = None


class stb_params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("T", ctypes.c_double), ("n_steps", ctypes.c_int32),
                ("quad_regular", ctypes.c_int32), ("quad_singular", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class stb_batch_item(ctypes.Structure):
    _fields_ = [("mesh", ctypes.c_void_p), ("params", stb_params), ("V", ctypes.c_void_p),
                ("K", ctypes.c_void_p)]


class StbError(RuntimeError):
    def __init__(self, code, where):
        lib = _library()
        msg = lib.stb_last_error_message().decode()
        super().__init__("%s: %s (%d): %s" % (where, lib.stb_status_string(code).decode(), code, msg))
        self.code = code


_P, _I32, _I64, _D, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
_PSZ = ctypes.POINTER(ctypes.c_size_t)
_PAR = ctypes.POINTER(stb_params)

_SIGS = {
    "stb_default_params": (stb_params, [_D, _D, _I32]),
    "stb_status_string": (ctypes.c_char_p, [_I32]),
    "stb_last_error_message": (ctypes.c_char_p, []),
    "stb_launch_count": (_I64, []),
    "stb_mesh_create": (_I32, [_P, _I64, _P, _I64, ctypes.POINTER(_P)]),
    "stb_mesh_destroy": (None, [_P]),
    "stb_mesh_info": (_I32, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "stb_assemble_workspace_size": (_I32, [_P, _PAR, _PSZ]),
    "stb_assemble": (_I32, [_P, _PAR, _P, _P, _P, _SZ, _P]),
    "stb_assemble_k1_workspace_size": (_I32, [_P, _PAR, _PSZ]),
    "stb_assemble_k1": (_I32, [_P, _PAR, _P, _P, _SZ, _P]),
    "stb_project_workspace_size": (_I32, [_P, _I32, _I32, _I32, _I32, _PSZ]),
    "stb_project_p1_workspace_size": (_I32, [_P, _PAR, _I32, _I32, _I32, _I32, _PSZ]),
    "stb_project_dirichlet_p1": (_I32, [_P, _PAR, _P, _I32, _I32, _I32, _I32, _P, _P, _SZ, _P]),
    "stb_rhs_p1_workspace_size": (_I32, [_P, _PAR, _I32, _PSZ]),
    "stb_assemble_d_workspace_size": (_I32, [_P, _PAR, _PSZ]),
    "stb_assemble_d": (_I32, [_P, _PAR, _P, _P, _P, _SZ, _P]),
    "stb_project_neumann": (_I32, [_P, _PAR, _P, _I32, _I32, _I32, _I32, _P, _P, _SZ, _P]),
    "stb_neumann_rhs_workspace_size": (_I32, [_P, _PAR, _I32, _PSZ]),
    "stb_neumann_rhs": (_I32, [_P, _PAR, _P, _P, _I32, _P, _P, _SZ, _P]),
    "stb_neumann_solve_workspace_size": (_I32, [_P, _PAR, _I32, _PSZ]),
    "stb_neumann_solve": (_I32, [_P, _PAR, _P, _P, _I32, _P, _P, _SZ, _P]),
    "stb_dirichlet_error_p1": (_I32, [_P, _PAR, _P, _I32, _I32, _P, _I32, _I32, _P, _P, _SZ, _P]),
    "stb_assemble_vrhs_workspace_size": (_I32, [_P, _PAR, _I32, _PSZ]),
    "stb_assemble_vrhs": (_I32, [_P, _PAR, _P, _P, _I32, _P, _P, _SZ, _P]),
    "stb_assemble_nu_workspace_size": (_I32, [_P, _PAR, _P, _PSZ]),
    "stb_assemble_nu_mixed_counts": (_I32, [_PAR, _P, _P, _P, _P]),
    "stb_assemble_nu": (_I32, [_P, _PAR, _P, _P, _P, _P, _SZ, _P]),
    "stb_matvec_nu": (_I32, [_P, _I64, _I32, _I32, _P, _P, _P]),
    "stb_solve_nu_workspace_size": (_I32, [_I64, _I32, _I32, _PSZ]),
    "stb_solve_nu": (_I32, [_P, _I64, _I32, _I32, _P, _P, _P, _SZ, _P]),
    "stb_project_nu_workspace_size": (_I32, [_P, _PAR, _I32, _I32, _I32, _I32, _PSZ]),
    "stb_project_dirichlet_nu": (_I32, [_P, _PAR, _P, _P, _I32, _I32, _I32, _I32, _P, _P, _SZ,
                                        _P]),
    "stb_neumann_error_nu": (_I32, [_P, _PAR, _P, _P, _I32, _I32, _P, _I32, _I32, _P, _P, _SZ,
                                    _P]),
    "stb_dirichlet_rhs_nu_workspace_size": (_I32, [_P, _PAR, _PSZ]),
    "stb_dirichlet_rhs_nu": (_I32, [_P, _PAR, _P, _P, _P, _I32, _P, _P, _SZ, _P]),
    "stb_potentials_workspace_size": (_I32, [_P, _PAR, _I32, _I64, _I32, _PSZ]),
    "stb_potentials": (_I32, [_P, _PAR, _P, _I64, _P, _P, _I32, _I32, _P, _P, _P, _SZ, _P]),
    "stb_potentials_grid_workspace_size": (_I32, [_P, _PAR, _I32, _I64, _I32, _PSZ]),
    "stb_potentials_grid": (_I32, [_P, _PAR, _P, _I64, _D, _P, _P, _I32, _I32, _P, _P, _P, _SZ,
                                   _P]),
    "stb_dirichlet_rhs_p1": (_I32, [_P, _PAR, _P, _P, _I32, _P, _P, _SZ, _P]),
    "stb_project_dirichlet": (_I32, [_P, _PAR, _P, _I32, _I32, _I32, _I32, _P, _P, _SZ, _P]),
    "stb_toeplitz_workspace_size": (_I32, [_I64, _I32, _I32, _PSZ]),
    "stb_toeplitz_matvec": (_I32, [_P, _I32, _I64, _I32, _I32, _P, _D, _P, _P, _SZ, _P]),
    "stb_toeplitz_matvec_static": (_I32, [_P, _I32, _I64, _I32, _I32, _P, _D, _P, _P]),
    "stb_toeplitz_ex_workspace_size": (_I32, [_I64, _I32, _I32, _I32, _PSZ]),
    "stb_toeplitz_matvec_ex": (_I32, [_P, _I32, _I64, _I32, _I32, _P, _D, _P, _I32, _P, _SZ, _P]),
    "stb_batch_workspace_size": (_I32, [_P, _I32, _PSZ]),
    "stb_batch_assemble": (_I32, [_P, _I32, _I32, _P, _SZ, _P]),
    "stb_batch_prepare": (_I32, [_P, _I32, _I32, _P, _SZ, _P]),
    "stb_batch_launch": (_I32, [_P, _I32, _I32, _P, _SZ, _P]),
    "stb_batch_tune": (_I32, [_P, _I32, _P, _SZ, _P, ctypes.POINTER(_I32)]),
    "stb_rhs_workspace_size": (_I32, [_P, _PAR, _I32, _PSZ]),
    "stb_dirichlet_rhs": (_I32, [_P, _PAR, _P, _P, _I32, _P, _P, _SZ, _P]),
    "stb_solve_workspace_size": (_I32, [_P, _PAR, _I32, _PSZ]),
    "stb_dirichlet_solve": (_I32, [_P, _PAR, _P, _P, _I32, _P, _P, _SZ, _P]),
    "stb_solve_report": (_I32, [_P, _P, ctypes.POINTER(_I32), ctypes.POINTER(_D)]),
    "stb_error_workspace_size": (_I32, [_P, _PAR, _I32, _I32, _I32, _I32, _PSZ]),
    "stb_neumann_error": (_I32, [_P, _PAR, _P, _I32, _I32, _P, _I32, _I32, _P, _P, _SZ, _P]),
    "stb_workspace_status": (_I32, [_P, _P]),
    "stb_selftest_bounded_wait": (_I32, [_P, _I64, _I32, _P, _SZ, _P]),
    "stb_selftest_grid_barrier": (_I32, [_I32, _I32, _I64, _P, _SZ, _P]),
    "stb_measure_peaks": (_I32, [ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_D), _P]),
    "stb_trace_enable": (_I32, [_I32]),
    "stb_trace_reset": (_I32, []),
    "stb_trace_read": (_I32, [_P, _I32, ctypes.POINTER(_I32)]),
}


class stb_trace_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


def library_path():
    return _build.LIB


def _library():
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError("CUDA library %s is not built; run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(code, where):
    if code != STB_OK:
        raise StbError(code, where)


def _ptr(t):
    """Device pointer of a torch tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _host_f64(a):
    """Host array and its pointer: a numpy array (copied to float64 if
    needed), or a CPU torch tensor of float64 (e.g. page-locked, for calls
    with STB_FLAG_NO_SYNC), passed as is."""
    if hasattr(a, "data_ptr"):
        if a.is_cuda or a.dtype.itemsize != 8 or not a.is_contiguous() or not a.is_floating_point():
            raise ValueError("expected a contiguous float64 CPU tensor")
        return a, ctypes.c_void_p(a.data_ptr())
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.c_void_p)


# ---- small helpers ------------------------------------------------------------
def stb_default_params(alpha, T, n_steps, quad_regular=3, quad_singular=4, precision=STB_PREC_FP64,
                       storage=STB_STORE_F64):
    p = _library().stb_default_params(alpha, T, n_steps)
    p.quad_regular, p.quad_singular = quad_regular, quad_singular
    p.precision, p.storage = precision, storage
    return p


def stb_launch_count():
    return int(_library().stb_launch_count())


class Mesh:
    """Owns an stb_mesh handle."""

    def __init__(self, nodes, tris):
        nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        tris = np.ascontiguousarray(tris, dtype=np.int32)
        h = ctypes.c_void_p()
        _check(_library().stb_mesh_create(nodes.ctypes.data_as(_P), nodes.shape[0],
                                          tris.ctypes.data_as(_P), tris.shape[0], ctypes.byref(h)),
               "stb_mesh_create")
        self.handle = h
        n, e, t = _I64(), _I64(), _I64()
        _check(_library().stb_mesh_info(h, ctypes.byref(n), ctypes.byref(e), ctypes.byref(t)),
               "stb_mesh_info")
        self.n_nodes, self.n_tris, self.n_touching = n.value, e.value, t.value

    def close(self):
        if self.handle:
            _library().stb_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stb_mesh_create(nodes, tris):
    return Mesh(nodes, tris)


def _size(fn, *args):
    n = _SZ()
    _check(fn(*args, ctypes.byref(n)), fn.__name__)
    return n.value


def stb_assemble_workspace_size(mesh, params):
    return _size(_library().stb_assemble_workspace_size, mesh.handle, ctypes.byref(params))


def stb_assemble(mesh, params, V, K, workspace, stream=None):
    _check(_library().stb_assemble(mesh.handle, ctypes.byref(params), _ptr(V), _ptr(K),
                                   _ptr(workspace), workspace.numel() * workspace.element_size(),
                                   _stream(stream)), "stb_assemble")


def stb_assemble_k1_workspace_size(mesh, params):
    return _size(_library().stb_assemble_k1_workspace_size, mesh.handle, ctypes.byref(params))


def stb_assemble_k1(mesh, params, K1, workspace, stream=None):
    _check(_library().stb_assemble_k1(mesh.handle, ctypes.byref(params), _ptr(K1), _ptr(workspace),
                                      workspace.numel() * workspace.element_size(),
                                      _stream(stream)), "stb_assemble_k1")


def stb_project_workspace_size(mesh, nrhs, n_src, q_space=8, n_time=16):
    return _size(_library().stb_project_workspace_size, mesh.handle, nrhs, n_src, q_space, n_time)


def stb_project_dirichlet(mesh, params, sources, g, workspace, q_space=8, n_time=16, stream=None):
    src, sp = _host_f64(sources)
    nrhs, n_src = src.shape[0], src.shape[1]
    _check(_library().stb_project_dirichlet(mesh.handle, ctypes.byref(params), sp, nrhs, n_src,
                                            q_space, n_time, _ptr(g), _ptr(workspace),
                                            workspace.numel() * workspace.element_size(),
                                            _stream(stream)), "stb_project_dirichlet")


def stb_project_p1_workspace_size(mesh, params, nrhs, n_src, q_space=8, n_time=16):
    return _size(_library().stb_project_p1_workspace_size, mesh.handle, ctypes.byref(params), nrhs,
                 n_src, q_space, n_time)


def stb_project_dirichlet_p1(mesh, params, sources, g1, workspace, q_space=8, n_time=16,
                             stream=None):
    src, sp = _host_f64(sources)
    nrhs, n_src = src.shape[0], src.shape[1]
    _check(_library().stb_project_dirichlet_p1(mesh.handle, ctypes.byref(params), sp, nrhs, n_src,
                                               q_space, n_time, _ptr(g1), _ptr(workspace),
                                               workspace.numel() * workspace.element_size(),
                                               _stream(stream)), "stb_project_dirichlet_p1")


def stb_rhs_p1_workspace_size(mesh, params, nrhs):
    return _size(_library().stb_rhs_p1_workspace_size, mesh.handle, ctypes.byref(params), nrhs)


def stb_dirichlet_rhs_p1(mesh, params, K1, g1, nrhs, f, workspace, stream=None):
    _check(_library().stb_dirichlet_rhs_p1(mesh.handle, ctypes.byref(params), _ptr(K1), _ptr(g1),
                                           nrhs, _ptr(f), _ptr(workspace),
                                           workspace.numel() * workspace.element_size(),
                                           _stream(stream)), "stb_dirichlet_rhs_p1")


def stb_potentials_workspace_size(mesh, params, nrhs, n_pts, q_space=4):
    return _size(_library().stb_potentials_workspace_size, mesh.handle, ctypes.byref(params), nrhs,
                 n_pts, q_space)


def stb_potentials(mesh, params, points, w, u1, nrhs, slp, dlp, workspace, q_space=4,
                   stream=None):
    """points: CUDA float64 [n_pts, 4]; w / u1 / slp / dlp: CUDA tensors or None."""
    _check(_library().stb_potentials(mesh.handle, ctypes.byref(params), _ptr(points),
                                     points.shape[0], _ptr(w), _ptr(u1), nrhs, q_space, _ptr(slp),
                                     _ptr(dlp), _ptr(workspace),
                                     workspace.numel() * workspace.element_size(),
                                     _stream(stream)), "stb_potentials")


def stb_potentials_grid_workspace_size(mesh, params, nrhs, n_pts, q_space=4):
    return _size(_library().stb_potentials_grid_workspace_size, mesh.handle, ctypes.byref(params),
                 nrhs, n_pts, q_space)


def stb_potentials_grid(mesh, params, points3, eps, w, u1, nrhs, slp, dlp, workspace, q_space=4,
                        stream=None):
    """points3: CUDA float64 [n_pts, 3]; slp / dlp: [nrhs, n_steps, n_pts] or None."""
    _check(_library().stb_potentials_grid(mesh.handle, ctypes.byref(params), _ptr(points3),
                                          points3.shape[0], eps, _ptr(w), _ptr(u1), nrhs, q_space,
                                          _ptr(slp), _ptr(dlp), _ptr(workspace),
                                          workspace.numel() * workspace.element_size(),
                                          _stream(stream)), "stb_potentials_grid")


def stb_assemble_d_workspace_size(mesh, params):
    return _size(_library().stb_assemble_d_workspace_size, mesh.handle, ctypes.byref(params))


def stb_assemble_d(mesh, params, V, D, workspace, stream=None):
    _check(_library().stb_assemble_d(mesh.handle, ctypes.byref(params), _ptr(V), _ptr(D),
                                     _ptr(workspace), workspace.numel() * workspace.element_size(),
                                     _stream(stream)), "stb_assemble_d")


def stb_project_neumann(mesh, params, sources, hd, workspace, q_space=8, n_time=16, stream=None):
    src, sp = _host_f64(sources)
    nrhs, n_src = src.shape[0], src.shape[1]
    _check(_library().stb_project_neumann(mesh.handle, ctypes.byref(params), sp, nrhs, n_src,
                                          q_space, n_time, _ptr(hd), _ptr(workspace),
                                          workspace.numel() * workspace.element_size(),
                                          _stream(stream)), "stb_project_neumann")


def stb_neumann_rhs_workspace_size(mesh, params, nrhs):
    return _size(_library().stb_neumann_rhs_workspace_size, mesh.handle, ctypes.byref(params), nrhs)


def stb_neumann_rhs(mesh, params, K1, hd, nrhs, f, workspace, stream=None):
    _check(_library().stb_neumann_rhs(mesh.handle, ctypes.byref(params), _ptr(K1), _ptr(hd), nrhs,
                                      _ptr(f), _ptr(workspace),
                                      workspace.numel() * workspace.element_size(),
                                      _stream(stream)), "stb_neumann_rhs")


def stb_neumann_solve_workspace_size(mesh, params, nrhs):
    return _size(_library().stb_neumann_solve_workspace_size, mesh.handle, ctypes.byref(params),
                 nrhs)


def stb_neumann_solve(mesh, params, D, f, nrhs, u, workspace, stream=None):
    _check(_library().stb_neumann_solve(mesh.handle, ctypes.byref(params), _ptr(D), _ptr(f), nrhs,
                                        _ptr(u), _ptr(workspace),
                                        workspace.numel() * workspace.element_size(),
                                        _stream(stream)), "stb_neumann_solve")


def stb_dirichlet_error_p1(mesh, params, sources, u1, out, workspace, q_space=8, n_time=16,
                           stream=None):
    src, sp = _host_f64(sources)
    nrhs, n_src = src.shape[0], src.shape[1]
    _check(_library().stb_dirichlet_error_p1(mesh.handle, ctypes.byref(params), sp, nrhs, n_src,
                                             _ptr(u1), q_space, n_time, _ptr(out), _ptr(workspace),
                                             workspace.numel() * workspace.element_size(),
                                             _stream(stream)), "stb_dirichlet_error_p1")


def stb_assemble_vrhs_workspace_size(mesh, params, nrhs):
    return _size(_library().stb_assemble_vrhs_workspace_size, mesh.handle, ctypes.byref(params),
                 nrhs)


def stb_assemble_vrhs(mesh, params, V, g, nrhs, f, workspace, stream=None):
    _check(_library().stb_assemble_vrhs(mesh.handle, ctypes.byref(params), _ptr(V), _ptr(g), nrhs,
                                        _ptr(f), _ptr(workspace),
                                        workspace.numel() * workspace.element_size(),
                                        _stream(stream)), "stb_assemble_vrhs")


# ---- non-uniform time grids -------------------------------------------------------
def _times(times):
    t, tp = _host_f64(times)
    return t, tp


def stb_assemble_nu_mixed_counts(params, times):
    """(closed-form evaluations, Gauss nodes, blocks with a closed-form part)
    of the mixed non-uniform tables (host only)."""
    t, tp = _times(times)
    out = [ctypes.c_int64(0) for _ in range(3)]
    _check(_library().stb_assemble_nu_mixed_counts(ctypes.byref(params), tp,
                                                   *[ctypes.byref(o) for o in out]),
           "stb_assemble_nu_mixed_counts")
    return tuple(int(o.value) for o in out)


def stb_assemble_nu_workspace_size(mesh, params, times):
    t, tp = _times(times)
    return _size(_library().stb_assemble_nu_workspace_size, mesh.handle, ctypes.byref(params), tp)


def stb_assemble_nu(mesh, params, times, V, K, workspace, stream=None):
    t, tp = _times(times)
    _check(_library().stb_assemble_nu(mesh.handle, ctypes.byref(params), tp, _ptr(V), _ptr(K),
                                      _ptr(workspace), workspace.numel() * workspace.element_size(),
                                      _stream(stream)), "stb_assemble_nu")


def stb_matvec_nu(A, E, n_steps, nrhs, x, y, stream=None):
    _check(_library().stb_matvec_nu(_ptr(A), E, n_steps, nrhs, _ptr(x), _ptr(y), _stream(stream)),
           "stb_matvec_nu")


def stb_solve_nu_workspace_size(E, n_steps, nrhs):
    return _size(_library().stb_solve_nu_workspace_size, E, n_steps, nrhs)


def stb_solve_nu(V, E, n_steps, nrhs, f, w, workspace, stream=None):
    _check(_library().stb_solve_nu(_ptr(V), E, n_steps, nrhs, _ptr(f), _ptr(w), _ptr(workspace),
                                   workspace.numel() * workspace.element_size(), _stream(stream)),
           "stb_solve_nu")


def stb_project_nu_workspace_size(mesh, params, nrhs, n_src, q_space=8, n_time=16):
    return _size(_library().stb_project_nu_workspace_size, mesh.handle, ctypes.byref(params), nrhs,
                 n_src, q_space, n_time)


def stb_project_dirichlet_nu(mesh, params, times, sources, g, workspace, q_space=8, n_time=16,
                             stream=None):
    t, tp = _times(times)
    src, sp = _host_f64(sources)
    _check(_library().stb_project_dirichlet_nu(mesh.handle, ctypes.byref(params), tp, sp,
                                               src.shape[0], src.shape[1], q_space, n_time,
                                               _ptr(g), _ptr(workspace),
                                               workspace.numel() * workspace.element_size(),
                                               _stream(stream)), "stb_project_dirichlet_nu")


def stb_neumann_error_nu(mesh, params, times, sources, w, out, workspace, q_space=8, n_time=16,
                         stream=None):
    t, tp = _times(times)
    src, sp = _host_f64(sources)
    _check(_library().stb_neumann_error_nu(mesh.handle, ctypes.byref(params), tp, sp, src.shape[0],
                                           src.shape[1], _ptr(w), q_space, n_time, _ptr(out),
                                           _ptr(workspace),
                                           workspace.numel() * workspace.element_size(),
                                           _stream(stream)), "stb_neumann_error_nu")


def stb_dirichlet_rhs_nu_workspace_size(mesh, params):
    return _size(_library().stb_dirichlet_rhs_nu_workspace_size, mesh.handle, ctypes.byref(params))


def stb_dirichlet_rhs_nu(mesh, params, times, K, g, nrhs, f, workspace, stream=None):
    t, tp = _times(times)
    _check(_library().stb_dirichlet_rhs_nu(mesh.handle, ctypes.byref(params), tp, _ptr(K), _ptr(g),
                                           nrhs, _ptr(f), _ptr(workspace),
                                           workspace.numel() * workspace.element_size(),
                                           _stream(stream)), "stb_dirichlet_rhs_nu")


def stb_toeplitz_workspace_size(E, n_steps, nrhs):
    return _size(_library().stb_toeplitz_workspace_size, E, n_steps, nrhs)


def stb_toeplitz_matvec(A, a_storage, E, n_steps, nrhs, x, beta, y, workspace, stream=None):
    _check(_library().stb_toeplitz_matvec(_ptr(A), a_storage, E, n_steps, nrhs, _ptr(x), beta, _ptr(y),
                                          _ptr(workspace),
                                          workspace.numel() * workspace.element_size(),
                                          _stream(stream)), "stb_toeplitz_matvec")


def stb_toeplitz_ex_workspace_size(E, n_steps, nrhs, arith):
    return _size(_library().stb_toeplitz_ex_workspace_size, E, n_steps, nrhs, arith)


def stb_toeplitz_matvec_ex(A, a_storage, E, n_steps, nrhs, x, beta, y, arith, workspace, stream=None):
    _check(_library().stb_toeplitz_matvec_ex(_ptr(A), a_storage, E, n_steps, nrhs, _ptr(x), beta,
                                             _ptr(y), arith, _ptr(workspace),
                                             workspace.numel() * workspace.element_size(),
                                             _stream(stream)), "stb_toeplitz_matvec_ex")


def stb_toeplitz_matvec_static(A, a_storage, E, n_steps, nrhs, x, beta, y, stream=None):
    _check(_library().stb_toeplitz_matvec_static(_ptr(A), a_storage, E, n_steps, nrhs, _ptr(x), beta,
                                                 _ptr(y), _stream(stream)),
           "stb_toeplitz_matvec_static")


def _batch_items(meshes, params, V, K):
    """ctypes array of stb_batch_item from lists (K entries may be None)."""
    n = len(meshes)
    arr = (stb_batch_item * n)()
    for i in range(n):
        arr[i].mesh = meshes[i].handle
        arr[i].params = params[i]
        arr[i].V = _ptr(V[i]).value
        arr[i].K = _ptr(K[i]).value if K[i] is not None else None
    return arr


def stb_batch_workspace_size(meshes, params, V, K):
    items = _batch_items(meshes, params, V, K)
    return _size(_library().stb_batch_workspace_size, items, len(meshes))


def stb_batch_assemble(meshes, params, V, K, tile, workspace, stream=None):
    items = _batch_items(meshes, params, V, K)
    _check(_library().stb_batch_assemble(items, len(meshes), tile, _ptr(workspace),
                                         workspace.numel() * workspace.element_size(),
                                         _stream(stream)), "stb_batch_assemble")


def stb_batch_prepare(meshes, params, V, K, tile, workspace, stream=None):
    items = _batch_items(meshes, params, V, K)
    _check(_library().stb_batch_prepare(items, len(meshes), tile, _ptr(workspace),
                                        workspace.numel() * workspace.element_size(),
                                        _stream(stream)), "stb_batch_prepare")


def stb_batch_launch(meshes, params, V, K, tile, workspace, stream=None):
    items = _batch_items(meshes, params, V, K)
    _check(_library().stb_batch_launch(items, len(meshes), tile, _ptr(workspace),
                                       workspace.numel() * workspace.element_size(),
                                       _stream(stream)), "stb_batch_launch")


def stb_batch_tune(meshes, params, V, K, workspace, stream=None):
    items = _batch_items(meshes, params, V, K)
    tile = _I32()
    _check(_library().stb_batch_tune(items, len(meshes), _ptr(workspace),
                                     workspace.numel() * workspace.element_size(), _stream(stream),
                                     ctypes.byref(tile)), "stb_batch_tune")
    return tile.value


def stb_rhs_workspace_size(mesh, params, nrhs):
    return _size(_library().stb_rhs_workspace_size, mesh.handle, ctypes.byref(params), nrhs)


def stb_dirichlet_rhs(mesh, params, K, g, nrhs, f, workspace, stream=None):
    _check(_library().stb_dirichlet_rhs(mesh.handle, ctypes.byref(params), _ptr(K), _ptr(g), nrhs,
                                        _ptr(f), _ptr(workspace),
                                        workspace.numel() * workspace.element_size(),
                                        _stream(stream)), "stb_dirichlet_rhs")


def stb_solve_workspace_size(mesh, params, nrhs):
    return _size(_library().stb_solve_workspace_size, mesh.handle, ctypes.byref(params), nrhs)


def stb_dirichlet_solve(mesh, params, V, f, nrhs, w, workspace, stream=None):
    _check(_library().stb_dirichlet_solve(mesh.handle, ctypes.byref(params), _ptr(V), _ptr(f), nrhs,
                                          _ptr(w), _ptr(workspace),
                                          workspace.numel() * workspace.element_size(),
                                          _stream(stream)), "stb_dirichlet_solve")


def stb_solve_report(workspace, stream=None):
    """(refinements, relative residual) of the last solve with this workspace."""
    it, res = _I32(), _D()
    _check(_library().stb_solve_report(_ptr(workspace), _stream(stream), ctypes.byref(it),
                                       ctypes.byref(res)), "stb_solve_report")
    return int(it.value), float(res.value)


def stb_error_workspace_size(mesh, params, nrhs, n_src, q_space=8, n_time=16):
    return _size(_library().stb_error_workspace_size, mesh.handle, ctypes.byref(params), nrhs, n_src,
                 q_space, n_time)


def stb_neumann_error(mesh, params, sources, w, out, workspace, q_space=8, n_time=16, stream=None):
    src, sp = _host_f64(sources)
    _check(_library().stb_neumann_error(mesh.handle, ctypes.byref(params), sp, src.shape[0],
                                        src.shape[1], _ptr(w), q_space, n_time, _ptr(out),
                                        _ptr(workspace),
                                        workspace.numel() * workspace.element_size(),
                                        _stream(stream)), "stb_neumann_error")


def stb_workspace_status(workspace, stream=None):
    _check(_library().stb_workspace_status(_ptr(workspace), _stream(stream)), "stb_workspace_status")


def stb_selftest_bounded_wait(probe, limit_ns, arrive, workspace, stream=None):
    _check(_library().stb_selftest_bounded_wait(_ptr(probe), int(limit_ns), 1 if arrive else 0,
                                                _ptr(workspace),
                                                workspace.numel() * workspace.element_size(),
                                                _stream(stream)), "stb_selftest_bounded_wait")


def stb_selftest_grid_barrier(n_cta, skip, limit_ns, workspace, stream=None):
    _check(_library().stb_selftest_grid_barrier(int(n_cta), int(skip), int(limit_ns),
                                                _ptr(workspace),
                                                workspace.numel() * workspace.element_size(),
                                                _stream(stream)), "stb_selftest_grid_barrier")


def stb_measure_peaks(stream=None):
    """(FP64 FMA/s, FP32 FMA/s, MUFU exp2/s) measured on the current device."""
    a, b, c = _D(), _D(), _D()
    _check(_library().stb_measure_peaks(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                        _stream(stream)), "stb_measure_peaks")
    return a.value, b.value, c.value


def stb_trace_enable(on=True):
    _check(_library().stb_trace_enable(1 if on else 0), "stb_trace_enable")


def stb_trace_reset():
    _check(_library().stb_trace_reset(), "stb_trace_reset")


def stb_trace_read():
    """{kernel name: (launches, total device ms)} since the last reset."""
    n = _I32()
    _check(_library().stb_trace_read(None, 0, ctypes.byref(n)), "stb_trace_read")
    buf = (stb_trace_entry * max(n.value, 1))()
    _check(_library().stb_trace_read(ctypes.cast(buf, _P), n.value, ctypes.byref(n)),
           "stb_trace_read")
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms))
            for i in range(n.value)}
