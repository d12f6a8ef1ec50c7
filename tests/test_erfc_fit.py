"""The FP32 erfc of the mixed potentials, erfc(x) = exp(-x^2) P(1/(1 + 0.7x))
with P of degree 11 fitted to the scaled complementary error function: the
coefficients are read from the CUDA source and evaluated as the kernel does
(FP32 Horner form, exp2 of -log2(e) x^2 in FP32), against SciPy's erfc.

Bounds (the source comment's): P within 3e-7 of exp(x^2) erfc(x) in FP32,
erfc within 4e-7 + 3e-7 x^2 relative (the second term the FP32 roundings
of -log2(e) x^2 and of the exp2) wherever erfc is a normal FP32 number.
The table itself must be the one the committed fit (fit_erfc.py beside the
package) produces.

NumPy's exp2 stands in for the hardware's ex2.approx here: the error of the
hardware instruction is covered only by the GPU tests of the mixed
potentials, which compare the kernels' level values with the FP64 oracle."""
import os
import re

import numpy as np
import pytest

scipy_special = pytest.importorskip("scipy.special")

SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), os.pardir, "paper_2102_09811_gb300",
                   "csrc", "stb_potentials.cu")


def coefficients():
    text = open(SRC).read()
    m = re.search(r"constexpr float c\[12\] = \{([^}]*)\}", text)
    assert m, "coefficient table not found"
    vals = [float(v.strip().rstrip("f")) for v in m.group(1).split(",") if v.strip()]
    assert len(vals) == 12
    return np.array(vals, dtype=np.float32)


def erfc_fit(x):
    c = coefficients()
    x = x.astype(np.float32)
    t = (np.float32(1) / (np.float32(0.7) * x + np.float32(1))).astype(np.float32)
    P = np.full_like(x, c[11])
    for k in range(10, -1, -1):
        P = (P * t + c[k]).astype(np.float32)
    e = np.exp2((np.float32(-1.4426950408889634) * x * x).astype(np.float32)).astype(np.float32)
    return (e * P).astype(np.float32), P


def test_scaled_polynomial_within_bound():
    x = np.linspace(0.0, 12.0, 120001)
    _, P = erfc_fit(x)
    ref = scipy_special.erfcx(x.astype(np.float32).astype(np.float64))
    assert np.max(np.abs(P / ref - 1.0)) <= 3e-7


def test_erfc_within_bound():
    x = np.linspace(0.0, 9.0, 90001)
    got, _ = erfc_fit(x)
    xs = x.astype(np.float32).astype(np.float64)
    ref = scipy_special.erfc(xs)
    normal = ref > np.finfo(np.float32).tiny
    rel = np.abs(got[normal] / ref[normal] - 1.0)
    assert np.all(rel <= 4e-7 + 3e-7 * xs[normal] ** 2), np.max(rel)


def test_special_values():
    got, _ = erfc_fit(np.array([0.0, 20.0]))
    assert abs(got[0] - 1.0) <= 3e-7
    assert got[1] == 0.0  # exp2 far below the FP32 range


def test_table_is_the_committed_fit():
    """The CUDA table is the fit script's output rounded to FP32 (relative
    1e-6 leaves room for another LAPACK's last bits), and that fit meets the
    bound by itself."""
    import importlib.util
    path = os.path.join(os.path.dirname(SRC), os.pardir, "fit_erfc.py")
    spec = importlib.util.spec_from_file_location("fit_erfc", path)
    fit_erfc = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(fit_erfc)
    c = fit_erfc.fit()
    src = coefficients().astype(np.float64)
    assert np.all(np.abs(c - src) <= 1e-6 * np.abs(src)), np.abs(c / src - 1).max()
    assert fit_erfc.max_rel_error_f32(c) <= 3e-7
