"""Host-side tables of the mixed-precision non-uniform assembly (Sec. 7;
reading of the overlap-weight forms): counts from the C ABI's host-only
query against what the construction fixes, without a GPU.

* uniform grid of n steps: one closed form for the diagonal blocks (H(h):
  one evaluation) and one for the blocks k = i + 1 (the uniform block 1:
  H(h), H(2h), H(h)), 2n - 1 blocks with a closed-form part, and per block
  distance d >= 2 one node list: Gauss-Legendre on [(d-1)h, dh] (ratio
  d - 1) and [dh, (d+1)h] (ratio d) with 6/4/3/2 nodes for ratios below
  2/16/96/above;
* a grid with all steps different: every diagonal and every k = i + 1 block
  its own closed form (1 and 3 evaluations);
* the counts depend on ratios of steps only (scaling the grid changes
  nothing).
"""
import numpy as np
import pytest

from paper_2102_09811_gb300 import capi


def counts(times, alpha=1.0):
    n = len(times) - 1
    p = capi.stb_default_params(alpha, float(times[-1]), n, precision=capi.STB_PREC_MIXED)
    return capi.stb_assemble_nu_mixed_counts(p, np.asarray(times, dtype=np.float64))


def gauss_nodes(ratio):
    return 6 if ratio < 2 else 4 if ratio < 16 else 3 if ratio < 96 else 2


@pytest.mark.parametrize("n", [1, 2, 3, 8, 40, 130])
def test_uniform_grid(n):
    terms, nodes, blocks = counts(np.arange(n + 1) / 64.0)
    assert blocks == n + (n - 1)
    assert terms == 1 + (3 if n > 1 else 0)
    assert nodes == sum(gauss_nodes(d - 1) + gauss_nodes(d) for d in range(2, n))


def test_all_steps_different():
    n = 9
    steps = 1.2 ** np.arange(n)
    t = np.concatenate([[0.0], np.cumsum(steps)])
    terms, nodes, blocks = counts(t)
    assert blocks == 2 * n - 1
    assert terms == n + 3 * (n - 1)
    assert nodes > 0


def test_scale_invariance():
    rng = np.random.default_rng(11)
    t = np.concatenate([[0.0], np.cumsum(rng.uniform(0.01, 1.0, size=12))])
    assert counts(t) == counts(t * 8.0) == counts(t, alpha=3.0)


def test_rejects_bad_grids():
    with pytest.raises(capi.StbError):
        counts(np.array([0.0, 0.5, 0.5, 1.0]))
    with pytest.raises(capi.StbError):
        counts(np.array([0.1, 0.5, 1.0]))
