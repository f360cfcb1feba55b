"""Near-patch evaluation on the device (ncs_eval at targets within 2.5 eps of a patch, such
as the paper's mean-first-passage-time maps on the sphere of radius 1 - eps/5, Section 9.2):
  * against the oracle's near-patch quadrature plus fine-grid far field
    (oracle/neareval.py) at r = 1 -+ eps/5 and 1 -+ eps/50, every target near some patch;
  * approaching a lone patch along the normal, the device potential tends to the on-patch
    value sum_k fhat_k q_k(y0) fixed by the one-patch equation (Section 8), linearly in the
    distance (the Richardson limit of two distances reproduces it)."""
import numpy as np
import pytest

from oracle import neareval as NE, operator as O, solve as S, zernike
from oracle.geometry import local_to_global
from oracle.kernels import EXTERIOR, INTERIOR
from paper_1906_04209_gb300 import layouts as L, ncs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS, K, NPAN, NORD, NTH = 0.05, 21, 6, 10, 28


@pytest.fixture(scope="module", autouse=True)
def _cuda(libncs):
    assert torch.cuda.is_available(), "GPU test without a GPU"
    torch.cuda.set_device(0)


def _ctx(mode, c):
    ctx = ncs.Context(EPS, mode, K, npan=NPAN, nord=NORD, ntheta_fine=NTH, id_tol=1e-13, method=ncs.METHOD_DIRECT)
    ctx.set_patches(c)
    return ctx


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
@pytest.mark.parametrize("frac", [5.0, 50.0])
def test_near_targets_match_oracle(mode, frac):
    N = 5
    c = L.uniform(N, EPS, L.rng(53, mode))
    pre = O.make_precompute(EPS, mode, K, npan=NPAN, nord=NORD, ntheta=NTH, with_id=False)
    fhat = S.dense_solve(O.dense_operator(pre, c), O.rhs(pre, N))
    sgn = 1.0 if mode == EXTERIOR else -1.0
    rng = np.random.default_rng(54)
    tg = []
    for j in range(N):
        for t0 in (0.2, 0.7, 0.98, 1.3, 2.2):
            y = local_to_global(c[j], np.array([t0 * EPS]), np.array([rng.uniform(0, 2 * np.pi)]))[0]
            tg.append(y * (1.0 + sgn * EPS / frac))
    tg = np.array(tg)
    ref = NE.mean_field_outputs(pre, c, fhat, tg)
    ctx = _ctx(mode, c)
    out = ctx.eval(tg, fhat)
    err = np.abs(out - ref).max() / np.abs(ref).max()
    print(f"mode {mode} r = 1 {'+' if sgn > 0 else '-'} eps/{frac:g}: max error {err:.2e} over {len(tg)} targets")
    assert err <= 1e-9


@pytest.mark.parametrize("mode,t0", [(INTERIOR, 0.5), (EXTERIOR, 0.9)])
def test_lone_patch_potential_tends_to_patch_values(mode, t0):
    c = np.array([[0.3, -0.2, 0.9]])
    c /= np.linalg.norm(c)
    ctx = _ctx(mode, c)
    f = np.random.default_rng(3).standard_normal(K)
    th0 = 1.0
    y0 = local_to_global(c[0], np.array([t0 * EPS]), np.array([th0]))[0]
    on = zernike.q_eval(K, np.array([t0]), np.array([th0]))[0] @ f
    sgn = -1.0 if mode == INTERIOR else 1.0
    d1, d2 = 1e-6, 1e-8
    x = np.stack([y0 * (1 + sgn * d1), y0 * (1 + sgn * d2)])
    out = ctx.eval(x, f)
    if mode == EXTERIOR:
        u = 1.0 - out
    else:
        Is = ctx.operator()["I"] @ f
        u = 1.0 + 3.0 * (-Is) * (out - (1.0 - np.sum(x * x, axis=1)) / 6.0)
    v1, v2 = u
    assert abs((v1 - on) / (v2 - on) / (d1 / d2) - 1.0) < 0.05
    limit = v2 + (v2 - v1) * d2 / (d1 - d2)
    assert abs(limit - on) <= 1e-8 * abs(on)


def test_target_on_a_patch_is_rejected():
    c = np.array([[0.0, 0.0, 1.0]])
    ctx = _ctx(INTERIOR, c)
    f = np.ones(K)
    y0 = local_to_global(c[0], np.array([0.5 * EPS]), np.array([0.3]))
    with pytest.raises(ncs.NcsError) as e:
        ctx.eval(y0, f)
    assert e.value.code == ncs.NCS_E_INPUT
