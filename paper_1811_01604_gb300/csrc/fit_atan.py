"""Coefficients of the arctangent polynomial used by angle_upper() in mpr_internal.cuh.

atan(x) on [0, 1] is written as x * P(x^2) with P of degree 7.  P is fitted by weighted
least squares on Chebyshev nodes, the weights refined by Lawson's iteration towards the
minimax (equal-ripple) fit of atan(x)/x.  Run: python fit_atan.py  -> prints the
coefficients (highest power first) and the maximum error of an FP32 Horner evaluation.
"""
import numpy as np

DEG = 7


def fit(deg=DEG, n=4000, iters=60):
    k = np.arange(n)
    x = 0.5 + 0.5 * np.cos(np.pi * (k + 0.5) / n)       # Chebyshev nodes on [0, 1]
    A = np.vstack([(x * x) ** j for j in range(deg + 1)]).T
    y = np.arctan(x) / x
    w = np.full(n, 1.0 / n)
    c = np.linalg.lstsq(A, y, rcond=None)[0]
    for _ in range(iters):                                 # Lawson: w <- w |r|, renormalised
        r = np.abs(A @ c - y)
        w = w * np.sqrt(r) + 1e-300
        w /= w.sum()
        sw = np.sqrt(w)
        c = np.linalg.lstsq(A * sw[:, None], y * sw, rcond=None)[0]
    return c                                               # lowest power first


def horner_f32(c, x):
    cf = np.asarray(c, np.float32)
    x = np.asarray(x, np.float32)
    t = (x * x).astype(np.float32)
    acc = np.full_like(x, cf[-1])
    for j in range(len(cf) - 2, -1, -1):
        acc = (acc * t + cf[j]).astype(np.float32)
    return (acc * x).astype(np.float32)


if __name__ == "__main__":
    c = fit()
    xs = np.linspace(0.0, 1.0, 400001)
    err = np.abs(horner_f32(c, xs).astype(np.float64) - np.arctan(xs)).max()
    for v in c[::-1]:
        print("%.9e" % np.float32(v))
    print("max |error| of the FP32 Horner evaluation on [0, 1]: %.2e" % err)
