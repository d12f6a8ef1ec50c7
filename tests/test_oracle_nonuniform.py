"""Pins of the oracle on non-uniform time grids (Sec. 7: the temporal
antiderivatives carry over to non-uniform grids; the matrices stay block
lower triangular but are no longer Toeplitz):

* on a uniform grid every block V^{k,i}, K^{k,i} equals the Toeplitz block
  of index k - i of the uniform assembly (eq. vd, eq. V0, eq. K_d, eq. K0);
* additivity in time: splitting one step of a grid in two, every block of
  the coarse grid is the sum of the fine blocks it covers (the fine block
  whose trial interval follows the test interval is zero by causality);
* a block depends only on the two intervals' lengths and distance: on a
  grid of alternating steps a, b (exact binary fractions) the block pattern
  repeats with period two;
* the forward substitution against a dense solve of the whole block lower-
  triangular system, and the non-uniform data/right-hand side/error
  functions against the uniform ones on a uniform grid.
Tolerances: 1e-11 relative per block (the four-corner combinations cancel
like the second differences of the uniform blocks).
"""
import math

import numpy as np
import pytest

import workloads


def _blocks_close(a, b, tol=1e-11):
    nrm = np.linalg.norm(b)
    return np.linalg.norm(a - b) <= tol * max(nrm, 1e-300)


@pytest.fixture(scope="module")
def mesh():
    return workloads.cube_mesh(2)


def test_uniform_grid_reproduces_toeplitz_blocks(orc, mesh):
    nodes, tris = mesh
    alpha, n = 0.8, 6
    times = np.arange(n + 1) * 0.125
    Vn, Kn = orc.assemble_nu(nodes, tris, alpha, times)
    V, K = orc.assemble(nodes, tris, alpha, times[-1], n)
    for k in range(n):
        for i in range(k + 1):
            b = orc.block_index(k, i)
            assert _blocks_close(Vn[b], V[k - i]), (k, i)
            assert _blocks_close(Kn[b], K[k - i]), (k, i)


def test_splitting_a_step_is_additive(orc, mesh):
    nodes, tris = mesh
    alpha = 1.1
    coarse = np.array([0.0, 0.125, 0.375, 0.5, 0.875])
    fine = np.array([0.0, 0.125, 0.25, 0.375, 0.5, 0.875])  # step 1 split at 0.25
    Vc, Kc = orc.assemble_nu(nodes, tris, alpha, coarse)
    Vf, Kf = orc.assemble_nu(nodes, tris, alpha, fine)
    # coarse step c covers fine steps cover[c]
    cover = {0: [0], 1: [1, 2], 2: [3], 3: [4]}
    for k in range(4):
        for i in range(k + 1):
            sv = sum(Vf[orc.block_index(kf, if_)] for kf in cover[k] for if_ in cover[i]
                     if kf >= if_)
            sk = sum(Kf[orc.block_index(kf, if_)] for kf in cover[k] for if_ in cover[i]
                     if kf >= if_)
            assert _blocks_close(sv, Vc[orc.block_index(k, i)]), (k, i)
            assert _blocks_close(sk, Kc[orc.block_index(k, i)]), (k, i)


def test_blocks_depend_on_lengths_and_distance_only(orc, mesh):
    nodes, tris = mesh
    steps = [0.125, 0.25] * 3
    times = np.concatenate([[0.0], np.cumsum(steps)])
    V, K = orc.assemble_nu(nodes, tris, 0.7, times)
    for k in range(4):
        for i in range(k + 1):
            assert np.array_equal(V[orc.block_index(k, i)], V[orc.block_index(k + 2, i + 2)])
            assert np.array_equal(K[orc.block_index(k, i)], K[orc.block_index(k + 2, i + 2)])


def test_forward_substitution_against_dense_solve(orc, mesh):
    nodes, tris = mesh
    times = np.array([0.0, 0.05, 0.15, 0.35, 0.5, 0.9])
    n, E = len(times) - 1, len(tris)
    V, _ = orc.assemble_nu(nodes, tris, 1.0, times)
    M = np.zeros((n * E, n * E))
    for k in range(n):
        for i in range(k + 1):
            M[k * E:(k + 1) * E, i * E:(i + 1) * E] = V[orc.block_index(k, i)]
    f = np.random.default_rng(0).normal(size=(2, n, E))
    w = orc.solve_nu(V, f)
    for r in range(2):
        wd = np.linalg.solve(M, f[r].reshape(-1)).reshape(n, E)
        assert np.linalg.norm(w[r] - wd) <= 1e-9 * np.linalg.norm(wd)
    assert np.allclose(orc.matvec_nu(V, w), f, rtol=0, atol=1e-10 * np.abs(f).max())


def test_nonuniform_pipeline_on_a_uniform_grid(orc, mesh):
    nodes, tris = workloads.cube_mesh(2)
    alpha, n = 1.0, 4
    times = np.arange(n + 1) * 0.125
    T = times[-1]
    src = workloads.point_source((1.4, 0.3, 1.6), t0=0.0)
    g = orc.project_dirichlet(nodes, tris, alpha, T, n, src)
    gn = orc.project_dirichlet_nu(nodes, tris, alpha, times, src)
    assert np.abs(g - gn).max() <= 1e-13 * np.abs(g).max()
    V, K = orc.assemble(nodes, tris, alpha, T, n)
    Vn, Kn = orc.assemble_nu(nodes, tris, alpha, times)
    area, _ = orc.triangle_geometry(nodes, tris)
    w = orc.dirichlet_solve(V, orc.dirichlet_rhs(area, K, g, T))
    wn = orc.solve_nu(Vn, orc.dirichlet_rhs_nu(area, Kn, times, gn))
    assert np.linalg.norm(w - wn) <= 1e-9 * np.linalg.norm(w)
    e2, r2 = orc.neumann_error(nodes, tris, alpha, T, n, src, w)
    e2n, r2n = orc.neumann_error_nu(nodes, tris, alpha, times, src, w)
    assert abs(e2 - e2n) <= 1e-12 * r2 and abs(r2 - r2n) <= 1e-12 * r2
