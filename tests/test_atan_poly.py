"""The update kernel's arctangent polynomial (q = atan(x)/pi on [0, 1]): its
coefficients are those the committed derivation produces, and its float32
evaluation stays within 2e-7 relative error of atan(x)/pi."""
import os
import re

import numpy as np

from paper_2404_02813_gb300 import atan_poly

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUH = os.path.join(ROOT, "paper_2404_02813_gb300", "csrc", "rsf_tiled.cuh")


def kernel_coefficients():
    src = open(CUH).read()
    body = src[src.index("constexpr float kAtanPi[9]"):]
    body = body[:body.index("};")]
    vals = [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    return np.array(vals[::-1], dtype=np.float32)  # the array runs from c8 down to c0 (Horner order)


def test_kernel_constants_match_the_derivation():
    c = atan_poly.coefficients().astype(np.float32)
    k = kernel_coefficients()
    assert k.shape == c.shape
    np.testing.assert_array_max_ulp(k, c, maxulp=2)  # BLAS rounding may differ between machines


def test_float32_relative_error():
    assert atan_poly.max_rel_error_f32(kernel_coefficients().astype(np.float64)) < 2e-7


def test_end_points():
    c = kernel_coefficients().astype(np.float64)
    p = lambda x: x * np.polyval(c[::-1], x * x)
    assert abs(p(1.0) - 0.25) < 1e-7            # atan(1)/pi
    assert abs(p(1e-3) / (np.arctan(1e-3) / np.pi) - 1) < 1e-7
