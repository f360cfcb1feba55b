"""The offset split of the float-float pair kernels (f2_split_grid / block_grid): with
q = 2^(e - 23), 2^e >= B >= |v| for every offset v of a block, the high word
hi = q * rint(v / q) is an FP32 number, the FP32 difference of two highs is exact, and
hi + float(v - hi) represents v to q 2^-25. Checked here in IEEE FP32/FP64 arithmetic
(round to nearest, as the device's sub.rn.f32x2) on seeded offsets, including the extreme
ones at +-B and offsets at B exactly a power of two."""
import numpy as np


def grid(B):
    e = np.frexp(B)[1]  # B = f 2^e, f in [1/2, 1)
    return np.ldexp(1.0, e - 23)


def split(v, q):
    hi = np.rint(v / q) * q
    return hi, (v - hi).astype(np.float32)


def test_high_words_subtract_exactly():
    rng = np.random.default_rng(7)
    for B in (2.0, 1.0, 0.75, 3.1e-3, 2.0 ** -7, 1e-5):
        v = rng.uniform(-B, B, 20000)
        v[:4] = (B, -B, np.nextafter(B, 0), -np.nextafter(B, 0))
        q = grid(np.abs(v).max())
        hi, lo = split(v, q)
        h32 = hi.astype(np.float32)
        assert np.array_equal(h32.astype(np.float64), hi)              # the high word is an FP32 number
        a, s = h32[: len(v) // 2], h32[len(v) // 2:]
        d32 = a - s                                                     # FP32 subtraction
        assert np.array_equal(d32.astype(np.float64), hi[: len(v) // 2] - hi[len(v) // 2:])
        # the representation error: |lo| <= q/2, rounded to FP32
        assert np.abs(lo).max() <= q / 2
        err = np.abs((hi + lo.astype(np.float64)) - v).max()
        assert err <= q * 2.0 ** -25


def test_offset_accuracy_relative_to_distance():
    """A pair's offset from the split parts: (hi_a - hi_s) exact, (lo_a - lo_s) rounded once
    to FP32. The error is at most q 2^-25 per split plus q 2^-24 for the rounded difference,
    i.e. <= q 2^-23 <= B 2^-45 (q <= 2B 2^-23): ~1.4e-13 of the distance for pairs B/5 apart."""
    rng = np.random.default_rng(8)
    B = 0.37
    a = rng.uniform(-0.5 * B, 0.5 * B, 20000)
    s = a + rng.choice([-1, 1], 20000) * rng.uniform(0.2 * B, 0.5 * B, 20000)
    q = grid(max(np.abs(a).max(), np.abs(s).max()))
    ha, la = split(a, q)
    hs, ls = split(s, q)
    d = (ha.astype(np.float32) - hs.astype(np.float32)).astype(np.float64) + (la - ls).astype(np.float64)
    err = np.abs(d - (a - s))
    assert err.max() <= q * 2.0 ** -23
    rel = err / np.abs(a - s)
    assert rel.max() <= B * 2.0 ** -45 / (0.2 * B)
    print(f"max error {err.max():.2e} (bound {q * 2.0 ** -23:.2e}), relative to the distance {rel.max():.2e}")
