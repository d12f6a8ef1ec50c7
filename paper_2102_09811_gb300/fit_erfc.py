"""Fit of the FP32 erfc used by the mixed-precision potential kernels.

erfc(x) = exp(-x^2) P(t), t = 1 / (1 + 0.7 x), x >= 0, with P a polynomial
of degree 11 in t approximating the scaled complementary error function
erfcx(x) = exp(x^2) erfc(x) in relative error on [0, 12].  The fit is a
weighted least-squares problem on 40,000 equispaced points, its weights
updated by Lawson's rule (w_i <- w_i |e_i|, normalised) for 20 passes, which
drives the least-squares solution towards the minimax one.  SciPy's erfcx is
the target.  The coefficients are rounded to FP32; in FP32 Horner form the
polynomial is then within 3e-7 of erfcx, the rounding of the Horner steps
(not the 1.3e-8 approximation error) setting that figure.

  python paper_2102_09811_gb300/fit_erfc.py

prints the table in the form the CUDA source holds (`constexpr float c[12]`
in csrc/stb_potentials.cu) and the FP32 error on a fine grid.
"""
import numpy as np

DEGREE = 11
X_MAX = 12.0
N_POINTS = 40000
LAWSON_PASSES = 20


def fit():
    """Coefficients c_0 .. c_11 (float64, before rounding) of P(t) = sum c_k t^k."""
    from scipy.special import erfcx

    x = np.linspace(0.0, X_MAX, N_POINTS)
    t = 1.0 / (1.0 + 0.7 * x)
    f = erfcx(x)
    V = np.vander(t, DEGREE + 1, increasing=True) / f[:, None]  # rows: P(t_i) / f_i
    w = np.ones_like(x)
    c = None
    for _ in range(LAWSON_PASSES + 1):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(V * sw[:, None], sw, rcond=None)
        e = np.abs(V @ c - 1.0)
        w = w * e
        w /= w.sum()
    return c


def horner_f32(c, x):
    """P(t(x)) evaluated as the kernel does: FP32 reciprocal of 1 + 0.7 x and
    FP32 Horner steps."""
    c = np.asarray(c, dtype=np.float32)
    x = np.asarray(x).astype(np.float32)
    t = (np.float32(1) / (np.float32(0.7) * x + np.float32(1))).astype(np.float32)
    P = np.full_like(x, c[-1])
    for k in range(len(c) - 2, -1, -1):
        P = (P * t + c[k]).astype(np.float32)
    return P


def max_rel_error_f32(c, n=120001):
    from scipy.special import erfcx

    x = np.linspace(0.0, X_MAX, n)
    ref = erfcx(x.astype(np.float32).astype(np.float64))
    return float(np.max(np.abs(horner_f32(c, x) / ref - 1.0)))


def c_table(c):
    vals = ["%.9e" % v for v in np.asarray(c, dtype=np.float32)]
    return "constexpr float c[%d] = {%s};" % (len(vals), ", ".join(v + "f" for v in vals))


if __name__ == "__main__":
    c = fit()
    print(c_table(c))
    print("max |P_f32 / erfcx - 1| on [0, %g]: %.3e" % (X_MAX, max_rel_error_f32(c)))
