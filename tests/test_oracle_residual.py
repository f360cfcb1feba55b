"""Pins of the patch residual diagnostic (eq. l2res, the relative L2 residual of the
multiple-scattering system on one patch): exact zero for a lone patch, the exact size of a
known perturbation, consistency with the discrete equations, and the spectral decay in
the Zernike degree M that the paper's convergence study reports."""
import numpy as np
import pytest

from oracle import operator as O, residual as R, solve as S, zernike
from oracle.kernels import EXTERIOR, INTERIOR
from paper_1906_04209_gb300 import layouts as L


def _pre(eps, mode, K):
    return O.make_precompute(eps, mode, K, npan=6, nord=10, ntheta=28, with_id=False)


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_lone_patch_residual_vanishes(mode):
    # N = 1: fhat = P 1 reproduces the constant 1 exactly (q_0 is constant and the sampling
    # grid integrates the span exactly), so S sigma - 1 = 0
    pre = _pre(0.1, mode, 10)
    c = np.array([[0.0, 0.0, 1.0]])
    fhat = pre.P @ np.ones(pre.Kstar)
    assert R.patch_residual(pre, c, fhat, 0) < 1e-14


@pytest.mark.parametrize("k,exact", [(0, True), (1, False), (4, False)])
def test_residual_of_a_known_perturbation(k, exact):
    # adding delta to fhat_k changes r by delta q_k: for q_0 = 1/sqrt(pi) the root mean
    # square is delta/sqrt(pi) exactly; for the others it is delta/sqrt(pi) up to the
    # curvature of the patch (sin t against t: relative O(eps^2))
    eps, delta = 0.1, 1e-3
    pre = _pre(eps, INTERIOR, 10)
    c = np.array([[0.0, 0.0, 1.0]])
    fhat = pre.P @ np.ones(pre.Kstar)
    fhat[k] += delta
    got = R.patch_residual(pre, c, fhat, 0)
    want = delta / np.sqrt(np.pi)
    if exact:
        assert abs(got - want) < 1e-12 * want
    else:
        assert abs(got - want) < eps * eps * want


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_residual_matches_the_discrete_equations(mode):
    # the solved fhat_0 is the discrete Zernike transform of 1 - u_0 at the Zernike nodes
    # (eq. opinteqnsdisc), with u_0 summed here on the fly and in the dense operator's
    # blocks there; the residual is then the part of 1 - u_0 outside the K modes
    eps, K, N = 0.08, 21, 4
    pre = _pre(eps, mode, K)
    c = L.uniform(N, eps, L.rng(31 + mode))
    fhat = S.dense_solve(O.dense_operator(pre, c), O.rhs(pre, N))
    g_z = 1.0 - R.incoming_on_patch(pre, c, fhat, 0, eps * pre.r_z, pre.th_z)
    coef = pre.P @ g_z
    assert np.abs(coef - fhat[:K]).max() < 1e-12
    t, th, dA = R.patch_grid(pre)
    g = 1.0 - R.incoming_on_patch(pre, c, fhat, 0, t, th)
    rr = zernike.q_eval(K, t / eps, th) @ coef - g
    rms = np.sqrt(np.sum(dA * rr * rr) / np.sum(dA))
    assert abs(rms - R.patch_residual(pre, c, fhat, 0)) < 1e-13
    assert rms > 0.0


def test_residual_decays_spectrally_in_M():
    # the paper's convergence study: the residual falls geometrically as the Zernike
    # degree M grows (the incoming field of well-separated patches is analytic on the patch)
    eps, N = 0.06, 5
    c = L.uniform(N, eps, L.rng(41))
    res = []
    for K in (6, 15, 28, 45):  # M = 2, 4, 6, 8
        pre = _pre(eps, INTERIOR, K)
        fhat = S.dense_solve(O.dense_operator(pre, c), O.rhs(pre, N))
        res.append(max(R.patch_residual(pre, c, fhat, i) for i in range(N)))
    res = np.array(res)
    assert np.all(res[1:] < res[:-1])
    assert res[-1] < 1e-3 * res[0]
