"""Coefficients of the arctangent polynomial used by the update kernel.

q = atan(x) / pi for x in [0, 1] is evaluated as x * P(x^2), P of degree 8,
whose coefficients minimise the maximum relative error of x * P(x^2) against
atan(x)/pi on [0, 1].  They are found by Lawson's algorithm (C. L. Lawson,
1961: iteratively reweighted least squares converging to the minimax
solution) on a dense Chebyshev-clustered grid, in double precision, then
rounded to float.

    python -m paper_2404_02813_gb300.atan_poly      # prints the C initialiser
"""
from __future__ import annotations

import numpy as np

DEGREE = 8


def _grid(n: int = 40001) -> np.ndarray:
    x = np.concatenate([np.cos(np.linspace(0.0, np.pi / 2, n)), np.linspace(0.0, 1.0, n)])
    return np.unique(x[x > 1e-6])


def coefficients(degree: int = DEGREE, iters: int = 300) -> np.ndarray:
    """c[0..degree], P(t) = sum c_k t^k, minimax relative error of x P(x^2) vs atan(x)/pi."""
    x = _grid()
    t = x * x
    f = np.arctan(x) / (np.pi * x)                 # target of P(t)
    A = np.vander(t, degree + 1, increasing=True) / f[:, None]   # rows: P(t)/f(t)
    w = np.full(t.shape, 1.0 / t.size)
    c = None
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(A * sw[:, None], sw, rcond=None)
        e = np.abs(A @ c - 1.0)
        w = w * e
        w /= w.sum()
    return c


def max_rel_error_f32(c: np.ndarray, n: int = 200001) -> float:
    """Maximum relative error of the float32 evaluation (Horner, fused) against atan(x)/pi."""
    x = np.linspace(1e-6, 1.0, n).astype(np.float32)
    cf = c.astype(np.float32)
    t = (x * x).astype(np.float32)
    p = np.full_like(t, cf[-1])
    for ck in cf[-2::-1]:
        p = (p.astype(np.float64) * t + ck).astype(np.float32)   # one rounding per step, like fmaf
    q = (x * p).astype(np.float32)
    ref = np.arctan(x.astype(np.float64)) / np.pi
    return float(np.max(np.abs(q.astype(np.float64) / ref - 1.0)))


if __name__ == "__main__":
    c = coefficients()
    print("// P(t), t = x^2, c[0] .. c[%d]; max rel. error (float32 evaluation) %.2e"
          % (DEGREE, max_rel_error_f32(c)))
    print("{" + ", ".join("%.9ef" % v for v in c.astype(np.float32)) + "}")
