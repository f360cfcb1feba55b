"""The FMA-pipe reciprocal square root of the FP32 pair kernels (rsqrt_newton_x2 in
csrc/device_common.cuh): Lomont's seed (bits 0x5f375a86 minus half the bits of x, "Fast
Inverse Square Root", 2003) and two Newton steps y <- y (3/2 - (x/2) y^2), evaluated here in
emulated FP32 (each operation rounded to single precision) over 60 decades of x: the relative
error is 4.7e-6 at most, which the FP32 products that use it for a share of their pairs
absorb (the tuner keeps a variant only if its product matches the float-float product to
2e-5). The device code itself is checked through those products (test_gpu_tune.py)."""
import numpy as np


def _f32(v):
    return np.asarray(v, dtype=np.float64).astype(np.float32)


def _newton(x, steps):
    x = _f32(x)
    y = (np.int32(0x5f375a86) - (x.view(np.int32) >> 1)).view(np.float32)
    nhx = _f32(np.float64(-0.5) * x)
    for _ in range(steps):
        t = _f32(nhx.astype(np.float64) * y)                   # (-x/2) y
        r = _f32(t.astype(np.float64) * y + 1.5)                # fma(t, y, 3/2)
        y = _f32(y.astype(np.float64) * r)
    return y


def test_seed_and_two_newton_steps():
    x = np.logspace(-30, 30, 200001)
    exact = 1.0 / np.sqrt(_f32(x).astype(np.float64))
    e0 = np.abs(_newton(x, 0) / exact - 1.0).max()
    e1 = np.abs(_newton(x, 1) / exact - 1.0).max()
    e2 = np.abs(_newton(x, 2) / exact - 1.0).max()
    assert 0.030 < e0 < 0.035            # the seed alone: ~3.4 %
    assert 1.6e-3 < e1 < 1.8e-3          # one step: Lomont's published 1.75e-3
    assert 3e-6 < e2 < 5e-6              # two steps: ~1.5 e1^2 = 4.6e-6
