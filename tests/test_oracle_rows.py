"""Pin of the oracle's plain-C sampler of the compressed sums (oracle/rows.c), the
reference of every large-N parity test: it must reproduce the Python restatement of
the same sums (Section 7.1, eq. Tmap: rho_j = T f_j, z_i(k) = sum_{j != i} sum_m
G(x^z_{i,k}, x_{j,pi(m)}) rho_{j,m}) at every (patch, node) output of a small layout,
including patches centred at both poles (the frame's fallback axis), in both modes.
The Python side is itself pinned against the dense operator of eq. opinteqnsdisc
(test_oracle_operator.py), so a transposed T index, a frame sign or a wrong kernel
sign in the C code fails here."""
import numpy as np
import pytest

from oracle import native, operator as O
from oracle.kernels import EXTERIOR, INTERIOR
from paper_1906_04209_gb300 import layouts as L


def _layout_with_poles(N, eps, seed):
    """N seeded uniform centres with the first two replaced by the poles (and any
    centre closer than 3 eps to a pole dropped)."""
    c = L.uniform(N + 6, eps, L.rng(91, seed))
    poles = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]])
    keep = [p for p in c if np.all(np.arccos(np.clip(poles @ p, -1, 1)) >= 3.0 * eps)]
    out = np.vstack([poles, np.array(keep)[: N - 2]])
    assert L.min_geodesic_separation(out) >= 3.0 * eps * (1 - 1e-12)
    return out


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_rows_equal_compressed_sums(small_pre, mode):
    eps = 0.05
    pre = small_pre(mode, eps=eps)
    N = 40
    c = _layout_with_poles(N, eps, mode)
    x = np.random.default_rng(40 + mode).standard_normal(N * pre.K)
    ref = O.id_field(pre, c, x)                      # (N, K*)
    patches = np.repeat(np.arange(N), pre.Kstar)
    nodes = np.tile(np.arange(pre.Kstar), N)
    got = native.rows(pre, c, x, patches, nodes).reshape(N, pre.Kstar)
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(got - ref).max() <= 1e-13 * scale
    # the pole patches see the field of the others in their own (fallback) frame
    assert np.abs(got[:2] - ref[:2]).max() <= 1e-13 * scale


def test_rows_single_patch_and_linearity(small_pre):
    """N = 1 has no other patch (zero field); the sums are linear in x."""
    pre = small_pre(INTERIOR)
    c1 = np.array([[0.0, 0.6, 0.8]])
    x1 = np.random.default_rng(3).standard_normal(pre.K)
    z = native.rows(pre, c1, x1, np.zeros(4, dtype=np.int64), np.arange(4))
    assert np.all(z == 0.0)
    N = 6
    c = L.uniform(N, pre.eps, L.rng(92))
    rng = np.random.default_rng(4)
    xa, xb = rng.standard_normal(N * pre.K), rng.standard_normal(N * pre.K)
    pt, nd = rng.integers(N, size=30), rng.integers(pre.Kstar, size=30)
    za = native.rows(pre, c, xa, pt, nd)
    zb = native.rows(pre, c, xb, pt, nd)
    zab = native.rows(pre, c, 2.0 * xa - 3.0 * xb, pt, nd)
    assert np.abs(zab - (2.0 * za - 3.0 * zb)).max() <= 1e-13 * np.abs(zab).max()
