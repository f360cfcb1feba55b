"""Pins of the one-patch solver (Sections 5 and 8) against a closed-form asymptotic
expansion and an off-grid residual check.

Small-eps expansion (derived here, not printed in the paper): with the kernel
2/d + s log(2/d) + O(d) (s = +1 interior, -1 exterior) and the flat-disk
(Weber) solution of int 2/d sigma = 1, I_0 = eps/pi, the constant part of the log
term resums to I = I_0 / (1 + s I_0 log(2/eps)) and the log-energy of the Weber
density gives the next term:
    (pi I / eps) (1 + s (eps/pi) log(2/eps)) = 1 - s (eps/pi) (3/2 - 2 log 2) + O(eps^2 log^2 eps),
where 3/2 - 2 log 2 = int int log(1/|xi - xi'|) dmu dmu' for the normalised Weber
measure dmu = dxi / (2 pi sqrt(1 - |xi|^2)) on the unit disk.
"""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import onepatch, zernike
from oracle.kernels import EXTERIOR, INTERIOR


def test_log_energy_constant():
    f = lambda r: -2 * np.log(r) * r / np.sqrt(1 - r * r) * (1 - np.sqrt(1 - r * r))
    assert abs(quad(f, 0, 1, limit=200)[0] - (1.5 - 2 * np.log(2))) < 1e-10


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
@pytest.mark.parametrize("eps,rtol", [(1e-3, 0.02), (1e-4, 0.003)])
def test_small_eps_expansion(mode, eps, rtol):
    op = onepatch.solve_one_patch(eps, mode, 1, npan=10, nord=12, ntheta=8)
    Is = op.I[0] * np.sqrt(np.pi)  # f = 1 has the single coefficient sqrt(pi) on q_1
    s = 1.0 if mode == INTERIOR else -1.0
    lhs = np.pi * Is / eps * (1 + s * eps / np.pi * np.log(2 / eps)) - 1.0
    rhs = -s * eps / np.pi * (1.5 - 2 * np.log(2))
    assert abs(lhs - rhs) < rtol * abs(rhs)


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_off_grid_residual(mode):
    """Residual of S b_j = q_j at points between the collocation nodes (the check
    behind eq. patcherrl2): small relative to |q_j|."""
    K = 10
    op = onepatch.solve_one_patch(0.05, mode, K, npan=8, nord=12, ntheta=16)
    rng = np.random.default_rng(3)
    t = np.sort(rng.uniform(0.02, 0.98, 6)) * 0.05
    th = rng.uniform(0, 2 * np.pi, 6)
    for j in (0, 1, 3, 5, 9):
        res = onepatch.one_patch_residual(op, j, t, th)
        rr, tt = np.meshgrid(np.linspace(0, 1, 20), np.linspace(0, 2 * np.pi, 21))
        scale = np.abs(zernike.q_eval(K, rr.ravel(), tt.ravel())[:, j]).max()
        assert np.abs(res).max() < 1e-9 * scale


def test_I_only_axisymmetric():
    """I = w^T B vanishes on every basis function with m > 0."""
    op = onepatch.solve_one_patch(0.1, INTERIOR, 21, npan=6, nord=10, ntheta=24)
    for j, (n, m, c) in enumerate(zernike.basis_list(21)):
        if m > 0:
            assert abs(op.I[j]) < 1e-14 * np.abs(op.I).max()
