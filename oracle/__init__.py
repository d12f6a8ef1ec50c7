"""FP64 CPU oracle of the space-time heat BEM hot path (TEST INFRASTRUCTURE).

A plain, slow, obviously correct C implementation (``orc_*.c``) of what the
GPU library computes: heat-kernel antiderivatives (Sec. 3), regular and
regularised spatial quadrature (eq. quad_reg, eq. quad_duffy), assembly of the
Toeplitz blocks V^d and K^d (Sec. 3.1-3.2, Sec. 5), Dirichlet data projection,
right-hand side, block-Toeplitz matvec, forward-substitution solve and the
L2(Sigma_h) error (Sec. 3.4, Sec. 6.1).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's cpu_baseline /
reference legs may import this package.  It shares no code with the CUDA
path; the product must never route through it.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against values fixed by the paper or by mathematics (closed forms, limits,
integral identities, invariants, brute-force quadrature).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

DISJOINT, VERTEX, EDGE, IDENTICAL = 0, 1, 2, 3

_D = ctypes.c_double
_I = ctypes.c_int
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_P = ctypes.c_void_p


def lib():
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            path = _build.build()
        L = ctypes.CDLL(path)
        for name in ("orc_heat_kernel", "orc_G_dtau", "orc_G_dtau_dt"):
            getattr(L, name).restype = _D
            getattr(L, name).argtypes = [_D, _D, _D]
        for name in ("orc_dn_heat_kernel", "orc_dn_G_dtau_dt", "orc_dn_G_dtau"):
            getattr(L, name).restype = _D
            getattr(L, name).argtypes = [_D, _D, _D, _D]
        L.orc_V_d.restype = _D
        L.orc_V_d.argtypes = [_D, _I, _D, _D]
        L.orc_K_d.restype = _D
        L.orc_K_d.argtypes = [_D, _D, _I, _D, _D]
        for name in ("orc_psi_series", "orc_psi_direct"):
            getattr(L, name).restype = _D
            getattr(L, name).argtypes = [_D]
        L.orc_gauss_legendre01.argtypes = [_I, _P, _P]
        L.orc_gauss_jacobi01.argtypes = [_I, _P, _P]
        L.orc_triangle_rule.argtypes = [_I, _P, _P, _P]
        L.orc_ss_rule_size.argtypes = [_I, _I]
        L.orc_ss_rule.argtypes = [_I, _I, _P, _P, _P, _P, _P]
        L.orc_triangle_geometry.argtypes = [_P, _I64, _P, _I64, _P, _P]
        L.orc_pair_class.argtypes = [_P, _P, _P, _P]
        L.orc_pair_sums.argtypes = [_P, _I64, _P, _I64, _I64, _I64, _D, _D,
                                    _I, _I, _I, _P, _P]
        L.orc_assemble_rows.argtypes = [_P, _I64, _P, _I64, _D, _D, _I32, _I32,
                                        _I32, _P, _I64, _P, _P, _P, _P]
        L.orc_project_dirichlet.argtypes = [_P, _I64, _P, _I64, _D, _D, _I32,
                                            _P, _I32, _I32, _I32, _I32, _P]
        L.orc_project_neumann.argtypes = [_P, _I64, _P, _I64, _D, _D, _I32,
                                          _P, _I32, _I32, _I32, _I32, _P]
        L.orc_toeplitz_matvec.argtypes = [_P, _I64, _I32, _I32, _P, _P]
        L.orc_dirichlet_rhs.argtypes = [_P, _P, _I64, _D, _I32, _I32, _P, _P]
        L.orc_dirichlet_solve.argtypes = [_P, _I64, _I32, _I32, _P, _P]
        L.orc_neumann_error.argtypes = [_P, _I64, _P, _I64, _D, _D, _I32, _P,
                                        _I32, _I32, _P, _I32, _I32, _P, _P]
        L.orc_assemble_k1_rows.argtypes = [_P, _I64, _P, _I64, _D, _D, _I32, _I32,
                                           _I32, _P, _I64, _P]
        L.orc_project_dirichlet_p1.argtypes = [_P, _I64, _P, _I64, _D, _D, _I32,
                                               _P, _I32, _I32, _I32, _I32, _P]
        L.orc_toeplitz_matvec_rect.argtypes = [_P, _I64, _I64, _I32, _I32, _P, _P]
        L.orc_assemble_d2_tris.argtypes = [_P, _I64, _P, _I64, _D, _D, _I32, _I32, _I32, _P,
                                           _I64, _P]
        L.orc_surface_curls.argtypes = [_P, _I64, _P, _I64, _P]
        L.orc_assemble_d1.argtypes = [_P, _I64, _P, _I64, _D, _I32, _P, _P]
        L.orc_neumann_rhs.argtypes = [_P, _P, _P, _I64, _I64, _D, _I32, _I32, _P, _P]
        L.orc_dirichlet_error_p1.argtypes = [_P, _I64, _P, _I64, _D, _D, _I32, _P, _I32, _I32,
                                             _P, _I32, _I32, _P, _P]
        L.orc_assemble_rows_nu.argtypes = [_P, _I64, _P, _I64, _D, _P, _I32, _I32, _I32, _P,
                                           _I64, _P, _P]
        L.orc_matvec_nu.argtypes = [_P, _I64, _I32, _I32, _P, _P]
        L.orc_solve_nu.argtypes = [_P, _I64, _I32, _I32, _P, _P]
        L.orc_project_dirichlet_nu.argtypes = [_P, _I64, _P, _I64, _D, _P, _I32, _P, _I32, _I32,
                                               _I32, _I32, _P]
        L.orc_dirichlet_rhs_nu.argtypes = [_P, _P, _I64, _P, _I32, _I32, _P, _P]
        L.orc_neumann_error_nu.argtypes = [_P, _I64, _P, _I64, _D, _P, _I32, _P, _I32, _I32, _P,
                                           _I32, _I32, _P, _P]
        L.orc_potentials.argtypes = [_P, _I64, _P, _I64, _D, _D, _I32, _P, _P, _I32, _P, _I64,
                                     _I32, _P, _P]
        L.orc_dirichlet_rhs_p1.argtypes = [_P, _P, _P, _I64, _I64, _D, _I32, _I32, _P, _P]
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("%s failed with code %d" % (what, rc))


# ---- kernels ---------------------------------------------------------------
def heat_kernel(rho, delta, alpha):
    return lib().orc_heat_kernel(rho, delta, alpha)


def dn_heat_kernel(rn, rho, delta, alpha):
    return lib().orc_dn_heat_kernel(rn, rho, delta, alpha)


def G_dtau(rho, delta, alpha):
    return lib().orc_G_dtau(rho, delta, alpha)


def G_dtau_dt(rho, delta, alpha):
    return lib().orc_G_dtau_dt(rho, delta, alpha)


def dn_G_dtau_dt(rn, rho, delta, alpha):
    return lib().orc_dn_G_dtau_dt(rn, rho, delta, alpha)


def dn_G_dtau(rn, rho, delta, alpha):
    return lib().orc_dn_G_dtau(rn, rho, delta, alpha)


def V_d(rho, d, h, alpha):
    return lib().orc_V_d(rho, d, h, alpha)


def K_d(rn, rho, d, h, alpha):
    return lib().orc_K_d(rn, rho, d, h, alpha)


def psi_series(x):
    return lib().orc_psi_series(x)


def psi_direct(x):
    return lib().orc_psi_direct(x)


# ---- quadrature --------------------------------------------------------------
def gauss_legendre01(n):
    x, w = np.zeros(n), np.zeros(n)
    _check(lib().orc_gauss_legendre01(n, _p(x), _p(w)), "gauss_legendre01")
    return x, w


def gauss_jacobi01(n):
    x, w = np.zeros(n), np.zeros(n)
    _check(lib().orc_gauss_jacobi01(n, _p(x), _p(w)), "gauss_jacobi01")
    return x, w


def triangle_rule(q):
    s1, s2, w = np.zeros(q * q), np.zeros(q * q), np.zeros(q * q)
    _check(lib().orc_triangle_rule(q, _p(s1), _p(s2), _p(w)), "triangle_rule")
    return s1, s2, w


def ss_rule(cls, m):
    n = lib().orc_ss_rule_size(cls, m)
    arrs = [np.zeros(n) for _ in range(5)]
    _check(lib().orc_ss_rule(cls, m, *[_p(a) for a in arrs]), "ss_rule")
    return tuple(arrs)


# ---- mesh ------------------------------------------------------------------
def triangle_geometry(nodes, tris):
    nodes, tris = _f64(nodes), _i32(tris)
    E = tris.shape[0]
    area, normal = np.zeros(E), np.zeros((E, 3))
    _check(lib().orc_triangle_geometry(_p(nodes), nodes.shape[0], _p(tris), E,
                                       _p(area), _p(normal)), "geometry")
    return area, normal


def pair_class(tl, tj):
    tl, tj = _i32(tl), _i32(tj)
    ol, oj = np.zeros(3, np.int32), np.zeros(3, np.int32)
    cls = lib().orc_pair_class(_p(tl), _p(tj), _p(ol), _p(oj))
    return cls, ol, oj


# ---- assembly --------------------------------------------------------------
def pair_sums(nodes, tris, l, j, alpha, h, n_levels, q_reg=3, m_ss=4):
    nodes, tris = _f64(nodes), _i32(tris)
    SV, SK = np.zeros(n_levels + 1), np.zeros(n_levels + 1)
    _check(lib().orc_pair_sums(_p(nodes), nodes.shape[0], _p(tris), tris.shape[0],
                               l, j, alpha, h, n_levels, q_reg, m_ss, _p(SV), _p(SK)),
           "pair_sums")
    return SV, SK


def assemble_rows(nodes, tris, alpha, T, n_steps, rows, q_reg=3, m_ss=4,
                  with_sums=False):
    """Rows of all blocks: V, K of shape [n_rows, n_steps, E]; with_sums also
    returns SV, SK of shape [n_rows, n_steps + 2, E] (levels 0..n_steps, then
    the delta = 0 singular sum)."""
    nodes, tris = _f64(nodes), _i32(tris)
    E = tris.shape[0]
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    nr = rows.shape[0]
    V = np.zeros((nr, n_steps, E))
    K = np.zeros((nr, n_steps, E))
    SV = np.zeros((nr, n_steps + 2, E)) if with_sums else None
    SK = np.zeros((nr, n_steps + 2, E)) if with_sums else None
    _check(lib().orc_assemble_rows(_p(nodes), nodes.shape[0], _p(tris), E, alpha, T,
                                   n_steps, q_reg, m_ss, _p(rows), nr, _p(V), _p(K),
                                   _p(SV) if with_sums else None,
                                   _p(SK) if with_sums else None), "assemble_rows")
    if with_sums:
        return V, K, SV, SK
    return V, K


def assemble(nodes, tris, alpha, T, n_steps, q_reg=3, m_ss=4):
    """All blocks in the library's layout [n_steps, E, E]."""
    E = np.asarray(tris).shape[0]
    V, K = assemble_rows(nodes, tris, alpha, T, n_steps, np.arange(E), q_reg, m_ss)
    return np.ascontiguousarray(V.transpose(1, 0, 2)), np.ascontiguousarray(K.transpose(1, 0, 2))


# ---- Dirichlet problem -------------------------------------------------------
def project_dirichlet(nodes, tris, alpha, T, n_steps, sources, q_space=8, n_time=16):
    """sources: [nrhs, n_src, 5] = (y1, y2, y3, t0, weight); g: [nrhs, n_steps, E]."""
    nodes, tris = _f64(nodes), _i32(tris)
    src = _f64(sources)
    nrhs, n_src = src.shape[0], src.shape[1]
    E = tris.shape[0]
    g = np.zeros((nrhs, n_steps, E))
    _check(lib().orc_project_dirichlet(_p(nodes), nodes.shape[0], _p(tris), E, alpha, T,
                                       n_steps, _p(src), n_src, nrhs, q_space, n_time,
                                       _p(g)), "project_dirichlet")
    return g


def project_neumann(nodes, tris, alpha, T, n_steps, sources, q_space=8, n_time=16):
    """Element means of the exact Neumann datum: [nrhs, n_steps, E]."""
    nodes, tris = _f64(nodes), _i32(tris)
    src = _f64(sources)
    nrhs, n_src = src.shape[0], src.shape[1]
    E = tris.shape[0]
    w = np.zeros((nrhs, n_steps, E))
    _check(lib().orc_project_neumann(_p(nodes), nodes.shape[0], _p(tris), E, alpha, T,
                                     n_steps, _p(src), n_src, nrhs, q_space, n_time,
                                     _p(w)), "project_neumann")
    return w


def toeplitz_matvec(A, x):
    A, x = _f64(A), _f64(x)
    n_steps, E = A.shape[0], A.shape[1]
    nrhs = x.shape[0]
    y = np.zeros_like(x)
    _check(lib().orc_toeplitz_matvec(_p(A), E, n_steps, nrhs, _p(x), _p(y)), "matvec")
    return y


def dirichlet_rhs(area, K, g, T):
    area, K, g = _f64(area), _f64(K), _f64(g)
    n_steps, E = K.shape[0], K.shape[1]
    f = np.zeros_like(g)
    _check(lib().orc_dirichlet_rhs(_p(area), _p(K), E, T, n_steps, g.shape[0],
                                   _p(g), _p(f)), "dirichlet_rhs")
    return f


def dirichlet_solve(V, f):
    V, f = _f64(V), _f64(f)
    n_steps, E = V.shape[0], V.shape[1]
    w = np.zeros_like(f)
    rc = lib().orc_dirichlet_solve(_p(V), E, n_steps, f.shape[0], _p(f), _p(w))
    if rc == -5:
        raise np.linalg.LinAlgError("V^0 is not positive definite")
    _check(rc, "dirichlet_solve")
    return w


def neumann_error(nodes, tris, alpha, T, n_steps, sources, w, q_space=8, n_time=16):
    """Returns (err2, ref2): squared L2(Sigma_h) norms summed over right-hand sides."""
    nodes, tris, src, w = _f64(nodes), _i32(tris), _f64(sources), _f64(w)
    e2, r2 = ctypes.c_double(0), ctypes.c_double(0)
    _check(lib().orc_neumann_error(_p(nodes), nodes.shape[0], _p(tris), tris.shape[0],
                                   alpha, T, n_steps, _p(src), src.shape[1], src.shape[0],
                                   _p(w), q_space, n_time, ctypes.byref(e2),
                                   ctypes.byref(r2)), "neumann_error")
    return e2.value, r2.value


# ---- piecewise-linear trial space in space (Sec. 3.2, Sec. 3.4) --------------
def assemble_k1_rows(nodes, tris, alpha, T, n_steps, rows, q_reg=3, m_ss=4):
    """Rows of the blocks of K_h with nodal hat trial functions:
    [n_rows, n_steps, n_nodes]."""
    nodes, tris = _f64(nodes), _i32(tris)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    K1 = np.zeros((rows.shape[0], n_steps, nodes.shape[0]))
    _check(lib().orc_assemble_k1_rows(_p(nodes), nodes.shape[0], _p(tris), tris.shape[0], alpha,
                                      T, n_steps, q_reg, m_ss, _p(rows), rows.shape[0], _p(K1)),
           "assemble_k1_rows")
    return K1


def assemble_k1(nodes, tris, alpha, T, n_steps, q_reg=3, m_ss=4):
    """All blocks of K_h (piecewise-linear trial): [n_steps, E, n_nodes]."""
    E = np.asarray(tris).shape[0]
    K1 = assemble_k1_rows(nodes, tris, alpha, T, n_steps, np.arange(E), q_reg, m_ss)
    return np.ascontiguousarray(K1.transpose(1, 0, 2))


def project_dirichlet_p1(nodes, tris, alpha, T, n_steps, sources, q_space=8, n_time=16):
    """L2 projection of the Dirichlet datum into X_h^{1,0}: [nrhs, n_steps, n_nodes]."""
    nodes, tris, src = _f64(nodes), _i32(tris), _f64(sources)
    nrhs, n_src = src.shape[0], src.shape[1]
    g1 = np.zeros((nrhs, n_steps, nodes.shape[0]))
    rc = lib().orc_project_dirichlet_p1(_p(nodes), nodes.shape[0], _p(tris), tris.shape[0],
                                        alpha, T, n_steps, _p(src), n_src, nrhs, q_space,
                                        n_time, _p(g1))
    if rc == -5:
        raise np.linalg.LinAlgError("p1 mass matrix is not positive definite")
    _check(rc, "project_dirichlet_p1")
    return g1


def toeplitz_matvec_rect(A, x):
    """A [n_steps, E, N], x [nrhs, n_steps, N] -> y [nrhs, n_steps, E]."""
    A, x = _f64(A), _f64(x)
    n_steps, E, N = A.shape
    y = np.zeros((x.shape[0], n_steps, E))
    _check(lib().orc_toeplitz_matvec_rect(_p(A), E, N, n_steps, x.shape[0], _p(x), _p(y)),
           "toeplitz_matvec_rect")
    return y


def dirichlet_rhs_p1(area, tris, K1, g1, T):
    """(1/2 M_h + K_h) g1 with the p0 x p1 mass: [nrhs, n_steps, E]."""
    area, tris, K1, g1 = _f64(area), _i32(tris), _f64(K1), _f64(g1)
    n_steps, E, N = K1.shape
    f = np.zeros((g1.shape[0], n_steps, E))
    _check(lib().orc_dirichlet_rhs_p1(_p(area), _p(tris), _p(K1), E, N, T, n_steps,
                                      g1.shape[0], _p(g1), _p(f)), "dirichlet_rhs_p1")
    return f


# ---- potentials: the discretised representation formula (Sec. 3.5) ----------
def potentials(nodes, tris, alpha, T, n_steps, points, w=None, u1=None, q=4):
    """Single-layer potential of w [nrhs, n_steps, E] (piecewise constant)
    and double-layer potential of u1 [nrhs, n_steps, n_nodes] (piecewise
    linear in space) at points [n_pts, 4] = (x1, x2, x3, t) off the
    boundary: (slp, dlp), each [nrhs, n_pts] or None."""
    nodes, tris, pts = _f64(nodes), _i32(tris), _f64(points)
    if w is None and u1 is None:
        raise ValueError("need w or u1")
    w = None if w is None else _f64(w)
    u1 = None if u1 is None else _f64(u1)
    nrhs = (w if w is not None else u1).shape[0]
    slp = np.zeros((nrhs, pts.shape[0])) if w is not None else None
    dlp = np.zeros((nrhs, pts.shape[0])) if u1 is not None else None
    _check(lib().orc_potentials(_p(nodes), nodes.shape[0], _p(tris), tris.shape[0], alpha, T,
                                n_steps, None if w is None else _p(w),
                                None if u1 is None else _p(u1), nrhs, _p(pts), pts.shape[0], q,
                                None if slp is None else _p(slp),
                                None if dlp is None else _p(dlp)), "potentials")
    return slp, dlp


# ---- hypersingular operator and the Neumann problem (Sec. 3.3, Sec. 3.4) ------
def assemble_d2(nodes, tris, alpha, T, n_steps, test_tris=None, q_reg=3, m_ss=4):
    """D^2 blocks [n_steps, N, N] from the pairs of the given test triangles
    (all by default) with every trial triangle."""
    nodes, tris = _f64(nodes), _i32(tris)
    E, N = tris.shape[0], nodes.shape[0]
    rows = np.arange(E) if test_tris is None else np.asarray(test_tris)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    D2 = np.zeros((n_steps, N, N))
    _check(lib().orc_assemble_d2_tris(_p(nodes), N, _p(tris), E, alpha, T, n_steps, q_reg, m_ss,
                                      _p(rows), rows.shape[0], _p(D2)), "assemble_d2_tris")
    return D2


def surface_curls(nodes, tris):
    """[E, 3, 3]: surface curl of the hat function of vertex v on triangle m."""
    nodes, tris = _f64(nodes), _i32(tris)
    out = np.zeros((tris.shape[0], 3, 3))
    _check(lib().orc_surface_curls(_p(nodes), nodes.shape[0], _p(tris), tris.shape[0], _p(out)),
           "surface_curls")
    return out


def assemble_d1(nodes, tris, alpha, V):
    """D^1 = T^T (alpha^2 V^d (x) I_3) T from V [n_steps, E, E]: [n_steps, N, N]."""
    nodes, tris, V = _f64(nodes), _i32(tris), _f64(V)
    n_steps, N = V.shape[0], nodes.shape[0]
    D1 = np.zeros((n_steps, N, N))
    _check(lib().orc_assemble_d1(_p(nodes), N, _p(tris), tris.shape[0], alpha, n_steps, _p(V),
                                 _p(D1)), "assemble_d1")
    return D1


def neumann_rhs(area, tris, K1, hd, T):
    """(1/2 M_h^{T_x} - K_h^{T_x}) h: [nrhs, n_steps, N]."""
    area, tris, K1, hd = _f64(area), _i32(tris), _f64(K1), _f64(hd)
    n_steps, E, N = K1.shape
    f = np.zeros((hd.shape[0], n_steps, N))
    _check(lib().orc_neumann_rhs(_p(area), _p(tris), _p(K1), E, N, T, n_steps, hd.shape[0],
                                 _p(hd), _p(f)), "neumann_rhs")
    return f


def dirichlet_error_p1(nodes, tris, alpha, T, n_steps, sources, u1, q_space=8, n_time=16):
    """(err2, ref2) of piecewise-linear Dirichlet data u1 [nrhs, n_steps, N]."""
    nodes, tris, src, u1 = _f64(nodes), _i32(tris), _f64(sources), _f64(u1)
    e2, r2 = ctypes.c_double(0), ctypes.c_double(0)
    _check(lib().orc_dirichlet_error_p1(_p(nodes), nodes.shape[0], _p(tris), tris.shape[0], alpha,
                                        T, n_steps, _p(src), src.shape[1], src.shape[0], _p(u1),
                                        q_space, n_time, ctypes.byref(e2), ctypes.byref(r2)),
           "dirichlet_error_p1")
    return e2.value, r2.value


# ---- non-uniform time grids (Sec. 7) -------------------------------------------
def n_blocks(n_steps):
    return n_steps * (n_steps + 1) // 2


def block_index(k, i):
    """Packed index of the block A^{k,i}, k >= i."""
    return k * (k + 1) // 2 + i


def assemble_rows_nu(nodes, tris, alpha, times, rows, q_reg=3, m_ss=4):
    """Rows of the blocks V^{k,i}, K^{k,i}: [n_rows, n_blocks, E] each."""
    nodes, tris, times = _f64(nodes), _i32(tris), _f64(times)
    n = times.shape[0] - 1
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    E = tris.shape[0]
    V = np.zeros((rows.shape[0], n_blocks(n), E))
    K = np.zeros_like(V)
    _check(lib().orc_assemble_rows_nu(_p(nodes), nodes.shape[0], _p(tris), E, alpha, _p(times), n,
                                      q_reg, m_ss, _p(rows), rows.shape[0], _p(V), _p(K)),
           "assemble_rows_nu")
    return V, K


def assemble_nu(nodes, tris, alpha, times, q_reg=3, m_ss=4):
    """All blocks [n_blocks, E, E] of V and K on the grid `times`."""
    E = np.asarray(tris).shape[0]
    V, K = assemble_rows_nu(nodes, tris, alpha, times, np.arange(E), q_reg, m_ss)
    return (np.ascontiguousarray(V.transpose(1, 0, 2)), np.ascontiguousarray(K.transpose(1, 0, 2)))


def matvec_nu(A, x):
    A, x = _f64(A), _f64(x)
    E, n = A.shape[1], x.shape[1]
    y = np.zeros_like(x)
    _check(lib().orc_matvec_nu(_p(A), E, n, x.shape[0], _p(x), _p(y)), "matvec_nu")
    return y


def solve_nu(V, f):
    V, f = _f64(V), _f64(f)
    w = np.zeros_like(f)
    rc = lib().orc_solve_nu(_p(V), V.shape[1], f.shape[1], f.shape[0], _p(f), _p(w))
    if rc == -5:
        raise np.linalg.LinAlgError("a diagonal block is not positive definite")
    _check(rc, "solve_nu")
    return w


def project_dirichlet_nu(nodes, tris, alpha, times, sources, q_space=8, n_time=16):
    nodes, tris, times, src = _f64(nodes), _i32(tris), _f64(times), _f64(sources)
    n = times.shape[0] - 1
    g = np.zeros((src.shape[0], n, tris.shape[0]))
    _check(lib().orc_project_dirichlet_nu(_p(nodes), nodes.shape[0], _p(tris), tris.shape[0],
                                          alpha, _p(times), n, _p(src), src.shape[1],
                                          src.shape[0], q_space, n_time, _p(g)),
           "project_dirichlet_nu")
    return g


def dirichlet_rhs_nu(area, K, times, g):
    area, K, times, g = _f64(area), _f64(K), _f64(times), _f64(g)
    f = np.zeros_like(g)
    _check(lib().orc_dirichlet_rhs_nu(_p(area), _p(K), K.shape[1], _p(times), g.shape[1],
                                      g.shape[0], _p(g), _p(f)), "dirichlet_rhs_nu")
    return f


def neumann_error_nu(nodes, tris, alpha, times, sources, w, q_space=8, n_time=16):
    nodes, tris, times, src, w = _f64(nodes), _i32(tris), _f64(times), _f64(sources), _f64(w)
    e2, r2 = ctypes.c_double(0), ctypes.c_double(0)
    _check(lib().orc_neumann_error_nu(_p(nodes), nodes.shape[0], _p(tris), tris.shape[0], alpha,
                                      _p(times), times.shape[0] - 1, _p(src), src.shape[1],
                                      src.shape[0], _p(w), q_space, n_time, ctypes.byref(e2),
                                      ctypes.byref(r2)), "neumann_error_nu")
    return e2.value, r2.value

