"""Pins of the Zernike basis and transform P (Section 4, Section 6)."""
from math import factorial

import numpy as np
import pytest

from oracle import zernike


def _radial_textbook(n, m, r):
    """Explicit finite-sum formula of the Zernike radial polynomial."""
    out = np.zeros_like(r)
    for s in range((n - m) // 2 + 1):
        c = (-1) ** s * factorial(n - s) / (factorial(s) * factorial((n + m) // 2 - s) * factorial((n - m) // 2 - s))
        out += c * r ** (n - 2 * s)
    return out


def test_radial_matches_textbook_sum():
    r = np.linspace(0, 1, 17)
    for n in range(0, 16):
        for m in range(n % 2, n + 1, 2):
            assert np.allclose(zernike.radial(n, m, r), _radial_textbook(n, m, r), atol=1e-10, rtol=0)
            assert abs(zernike.radial(n, m, np.array([1.0]))[0] - 1.0) < 1e-12


@pytest.mark.parametrize("K", [1, 10, 55, 64, 128, 136])
def test_transform_left_inverse(K):
    """P Q_z = I_K: the sampling rule is exact on the span (Section 4)."""
    P, _, _ = zernike.transform(K)
    Q = zernike.synthesis(K)
    assert np.abs(P @ Q - np.eye(K)).max() < 1e-12


def test_orthonormal_independent_rule():
    """Orthonormality (eq. zorthog normalisation) on a much finer independent grid."""
    K = 66
    x, w = np.polynomial.legendre.leggauss(40)
    r = 0.5 * (x + 1)
    nth = 64
    th = 2 * np.pi * np.arange(nth) / nth
    R, TH = np.meshgrid(r, th, indexing="ij")
    W = (0.5 * w * r)[:, None] * np.full(nth, 2 * np.pi / nth)[None, :]
    Q = zernike.q_eval(K, R.ravel(), TH.ravel())
    G = (Q * W.ravel()[:, None]).T @ Q
    assert np.abs(G - np.eye(K)).max() < 1e-12


def test_truncation_sets():
    """K = (M+1)(M+2)/2 gives 0 <= m <= n <= M; K = 64, 128 end on full cos/sin pairs."""
    b = zernike.basis_list(136)
    assert max(n for n, _, _ in b) == 15 and len({(n, m, c) for n, m, c in b}) == 136
    b64 = zernike.basis_list(64)
    assert sorted({(n, m) for n, m, _ in b64 if n == 10}) == [(10, 0), (10, 2), (10, 4), (10, 6), (10, 8)]
    b128 = zernike.basis_list(128)
    assert sorted({(n, m) for n, m, _ in b128 if n == 15}) == [(15, 1), (15, 3), (15, 5), (15, 7)]
    for bl in (b64, b128):
        for n, m, c in bl:
            if m > 0:
                assert (n, m, 1 - c) in bl
    assert zernike.sampling_nodes(15)[0].size == 16 * 31
