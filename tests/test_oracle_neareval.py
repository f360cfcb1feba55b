"""Pins of the oracle's near-patch evaluation of the single-layer potential
(oracle/neareval.py; off-surface Green's functions eqs. Gextoffsurface / Gintoffsurface):
the rewritten kernel equals the printed one, the direct quadrature equals the fine-grid sum
where the latter is accurate, and at points approaching the patch the potential tends to
its on-surface values, which the one-patch equation fixes (S b_k = q_k, Section 8)."""
import numpy as np
import pytest

from oracle import neareval as NE, operator as O, zernike
from oracle.geometry import local_to_global, patch_points
from oracle.kernels import EXTERIOR, INTERIOR, G_off_surface


def _pre(mode):
    return O.make_precompute(0.05, mode, 21, npan=6, nord=10, ntheta=28, with_id=False)


def _centre():
    c = np.array([0.3, -0.2, 0.9])
    return c / np.linalg.norm(c)


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_stable_kernel_equals_printed_form(mode):
    rng = np.random.default_rng(5)
    y = rng.standard_normal((2000, 3))
    y /= np.linalg.norm(y, axis=1)[:, None]
    x = rng.standard_normal((2000, 3))
    x /= np.linalg.norm(x, axis=1)[:, None]
    r = 1.0 + rng.uniform(0.0, 0.5, 2000) if mode == EXTERIOR else rng.uniform(0.2, 1.0, 2000)
    x *= r[:, None]
    keep = np.linalg.norm(x - y, axis=1) > 0.1
    a, b = NE.G_off_stable(x[keep], y[keep], mode), G_off_surface(x[keep], y[keep], mode)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_near_quadrature_equals_fine_grid_where_both_hold(mode):
    # 3 eps from the centre, eps/5 off the sphere: the fine grid is accurate there
    pre = _pre(mode)
    c, eps = _centre(), pre.eps
    f = np.random.default_rng(3).standard_normal(pre.K)
    y0 = local_to_global(c, np.array([3 * eps]), np.array([0.7]))[0]
    x = y0 * (1 - eps / 5 if mode == INTERIOR else 1 + eps / 5)
    fine = patch_points(c[None], pre.op.t_f, pre.op.th_f)[0]
    far = G_off_surface(x[None, :], fine, mode) @ (pre.op.w * (pre.op.B @ f))
    assert abs(NE.near_potential(pre, c, f, x) - far) <= 1e-10 * abs(far)


@pytest.mark.parametrize("mode,t0", [(INTERIOR, 0.5), (INTERIOR, 0.9), (EXTERIOR, 0.9)])
def test_near_potential_tends_to_the_patch_values(mode, t0):
    # approaching y0 on the patch along the normal the potential converges linearly in the
    # distance delta (the normal derivative jumps across the patch); the Richardson limit
    # of delta = 1e-6 and 1e-8 reproduces sum_k fhat_k q_k(y0)
    pre = _pre(mode)
    c, eps = _centre(), pre.eps
    f = np.random.default_rng(3).standard_normal(pre.K)
    th0 = 1.0
    y0 = local_to_global(c, np.array([t0 * eps]), np.array([th0]))[0]
    on = zernike.q_eval(pre.K, np.array([t0]), np.array([th0]))[0] @ f
    sgn = -1.0 if mode == INTERIOR else 1.0
    d1, d2 = 1e-6, 1e-8
    v1 = NE.near_potential(pre, c, f, y0 * (1 + sgn * d1))
    v2 = NE.near_potential(pre, c, f, y0 * (1 + sgn * d2))
    ratio = (v1 - on) / (v2 - on)
    assert abs(ratio / (d1 / d2) - 1.0) < 0.05
    limit = v2 + (v2 - v1) * d2 / (d1 - d2)
    assert abs(limit - on) <= 1e-8 * abs(on)


def test_mfpt_at_a_patch_tends_to_the_residual():
    # interior, a solved layout: approaching a patch, vbar = (v - 1)/(3 D) + (1 - |x|^2)/6
    # tends to r(y0)/(3 D), r the residual of the system there (eq. l2res), D = -I_sigma;
    # the near quadrature of the own patch and the residual's Zernike sum agree in the limit
    from oracle import residual as R, solve as S
    from paper_1906_04209_gb300 import layouts as L
    pre = _pre(INTERIOR)
    eps, N = pre.eps, 4
    c = L.uniform(N, eps, L.rng(52))
    fhat = S.dense_solve(O.dense_operator(pre, c), O.rhs(pre, N))
    t0, th0 = 0.5 * eps, 1.0
    y0 = local_to_global(c[0], np.array([t0]), np.array([th0]))[0]
    d1, d2 = 1e-6, 1e-8
    v1, v2 = NE.mean_field_outputs(pre, c, fhat, np.stack([y0 * (1 - d1), y0 * (1 - d2)]))
    limit = v2 + (v2 - v1) * d2 / (d1 - d2)
    Is = pre.op.I @ fhat.reshape(N, pre.K).sum(axis=0)
    r0 = R.residual_values(pre, c, fhat, 0, np.array([t0]), np.array([th0]))[0]
    assert abs(limit - r0 / (3.0 * -Is)) <= 1e-8
    assert abs(limit) < 1e-3
