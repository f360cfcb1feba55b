"""The patch residual of eq. l2res on the device (ncs_patch_residual) against the oracle's
(oracle/residual.py): the same discrete solution, the other patches' potential from the
compressed skeletons on the device and from the fine-grid quadrature in the oracle."""
import numpy as np
import pytest

from oracle import operator as O, residual as R, solve as S
from oracle.kernels import EXTERIOR, INTERIOR
from paper_1906_04209_gb300 import layouts as L, ncs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda(libncs):
    assert torch.cuda.is_available(), "GPU test without a GPU"
    torch.cuda.set_device(0)


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_patch_residual_matches_oracle(mode):
    eps, K, N = 0.06, 15, 5
    pre = O.make_precompute(eps, mode, K, npan=6, nord=10, ntheta=28, tau=1e-12)
    c = L.uniform(N, eps, L.rng(41))
    fhat = S.dense_solve(O.dense_operator(pre, c), O.rhs(pre, N))
    ctx = ncs.Context(eps, mode, K, operator=(pre.idr.T, pre.idr.t_skel, pre.idr.th_skel, pre.op.I),
                      method=ncs.METHOD_DIRECT)
    ctx.set_patches(c)
    for i in range(N):
        lib = ctx.patch_residual(i, fhat)
        ref = R.patch_residual(pre, c, fhat, i)
        # the skeletons reproduce the fine-grid far field to ~1e-12 of the field itself
        assert abs(lib - ref) <= 1e-10 + 1e-3 * ref, (i, lib, ref)


def test_patch_residual_lone_patch_and_errors():
    eps, K = 0.1, 10
    pre = O.make_precompute(eps, INTERIOR, K, npan=6, nord=10, ntheta=24, tau=1e-11)
    ctx = ncs.Context(eps, INTERIOR, K, operator=(pre.idr.T, pre.idr.t_skel, pre.idr.th_skel, pre.op.I),
                      method=ncs.METHOD_DIRECT)
    ctx.set_patches([[0.0, 0.0, 1.0]])
    fhat = pre.P @ np.ones(pre.Kstar)
    assert ctx.patch_residual(0, fhat) < 1e-14
    with pytest.raises(ncs.NcsError) as e:
        ctx.patch_residual(1, fhat)
    assert e.value.code == ncs.NCS_E_INPUT
