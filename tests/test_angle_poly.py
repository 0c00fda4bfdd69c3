"""The upper-half-plane arctangent of the CUDA path (angle_upper in mpr_internal.cuh), used
for the equilibrium angle sums and the state read-out.

Pins: the coefficients in the header are the ones csrc/fit_atan.py derives (least squares
on Chebyshev nodes, Lawson-refined); the FP32 evaluation of the same reduction and
polynomial stays within 4e-7 rad of numpy's arctan2 over the closed upper half circle,
including the axes, the diagonal and the end points.  The device function itself is pinned
on the GPU by the single-sweep parity tests, which read the state through it.
"""
import os
import re
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1811_01604_gb300", "csrc")


def header_coeffs():
    src = open(os.path.join(CSRC, "mpr_internal.cuh")).read()
    body = src[src.index("float angle_upper("):src.index("float a = p * x;")]
    return [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]


def fit_module():
    sys.path.insert(0, CSRC)
    try:
        import fit_atan
    finally:
        sys.path.pop(0)
    return fit_atan


def angle_upper_f32(c, s, coeffs):
    c = np.asarray(c, np.float32)
    s = np.asarray(s, np.float32)
    ac = np.abs(c)
    lo, hi = np.minimum(ac, s), np.maximum(ac, s)
    x = np.where(hi > 0, lo / np.where(hi > 0, hi, 1), 0).astype(np.float32)
    t = (x * x).astype(np.float32)
    p = np.full_like(x, np.float32(coeffs[0]))
    for cf in coeffs[1:]:
        p = (p * t + np.float32(cf)).astype(np.float32)
    a = (p * x).astype(np.float32)
    a = np.where(s > ac, np.float32(np.pi / 2) - a, a).astype(np.float32)
    return np.where(c < 0, np.float32(np.pi) - a, a).astype(np.float32)


def test_header_coefficients_are_the_fit():
    got = header_coeffs()
    want = [float("%.9e" % np.float32(v)) for v in fit_module().fit()[::-1]]
    assert len(got) == 8 and np.allclose(got, want, rtol=0, atol=0)


def test_reduction_and_polynomial_error_bound():
    coeffs = header_coeffs()
    rng = np.random.default_rng(7)
    th = np.concatenate([rng.uniform(0, np.pi, 1_000_000),
                         [0.0, np.pi / 4, np.pi / 2, 3 * np.pi / 4, np.pi],
                         np.pi / 4 + np.linspace(-1e-6, 1e-6, 101)])
    c, s = np.cos(th).astype(np.float32), np.maximum(np.sin(th), 0).astype(np.float32)
    exact = np.arctan2(s.astype(np.float64), c.astype(np.float64))
    err = np.abs(angle_upper_f32(c, s, coeffs).astype(np.float64) - exact)
    assert err.max() < 4e-7, err.max()
    assert angle_upper_f32(0.0, 0.0, coeffs) == 0.0
