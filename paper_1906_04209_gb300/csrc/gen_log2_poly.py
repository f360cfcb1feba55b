"""Coefficients of the FP32 log2 polynomial used by the pair kernels (lg2_poly in
device_common.cuh).

log2(1 + f) = f * P(f) on f in [sqrt(1/2) - 1, sqrt(2) - 1), P of degree 8, fitted by
linear least squares at 4000 Chebyshev points of that interval and rounded to FP32.
Run: python gen_log2_poly.py  (prints the C initialisers and the FP32 evaluation error).
"""
import numpy as np

DEG = 9  # terms f^1 .. f^9


def fit():
    lo, hi = np.sqrt(0.5) - 1.0, np.sqrt(2.0) - 1.0
    t = np.cos(np.pi * (np.arange(4000) + 0.5) / 4000)
    f = lo + (hi - lo) * (t + 1) / 2
    A = np.vstack([f ** (k + 1) for k in range(DEG)]).T
    c, *_ = np.linalg.lstsq(A, np.log2(1 + f), rcond=None)
    return c.astype(np.float32)


def eval32(c, x):
    """The kernel's evaluation, step for step, in FP32 (numpy)."""
    x = np.asarray(x, dtype=np.float32)
    i = x.view(np.int32)
    e = (i - np.int32(0x3F3504F3)) >> 23
    m = (i - (e << 23)).view(np.float32)
    f = m - np.float32(1)
    p = np.full_like(f, c[DEG - 1])
    for k in range(DEG - 2, -1, -1):
        p = (p * f + c[k]).astype(np.float32)
    return (f * p + e.astype(np.float32)).astype(np.float32)


if __name__ == "__main__":
    c = fit()
    x = np.exp(np.linspace(np.log(1e-6), np.log(1e6), 2_000_001)).astype(np.float32)
    err = np.abs(eval32(c, x).astype(np.float64) - np.log2(x.astype(np.float64))).max()
    print("// max |error| over [1e-6, 1e6]: %.2e" % err)
    print(", ".join("%.9ef" % v for v in c))
