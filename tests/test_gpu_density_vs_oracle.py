"""Solution densities against the oracle's FP64 solve (the error bars the solver targets: density
relative error <= 1e-6 for the mixed solve, <= 1e-10 in FP64): the oracle runs its own
GMRES (modified Gram-Schmidt, Section 7 Step 3 reading) on the compressed product of
Section 7.1 evaluated at every Zernike node by its plain-C sums, for the interior
workload's patch (eps = 0.02, K = 128) on a 120-patch layout (82 grid groups on 6 tree
levels). The library takes the same compressed operator, and solves with the direct and
the tree products in every precision; each error is printed as a number."""
import numpy as np
import pytest

from oracle import native, operator as O, solve as S
from oracle.kernels import EXTERIOR, INTERIOR
from paper_1906_04209_gb300 import layouts as L, ncs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda(libncs):
    assert torch.cuda.is_available(), "GPU test without a GPU"
    torch.cuda.set_device(0)


def _oracle_solution(pre, c):
    N = len(c)
    pt = np.repeat(np.arange(N), pre.Kstar)
    nd = np.tile(np.arange(pre.Kstar), N)

    def matvec(x):
        z = native.rows(pre, c, x, pt, nd).reshape(N, pre.Kstar)
        return x + (z @ pre.P.T).ravel()

    x, it, _, true = S.gmres(matvec, O.rhs(pre, N), 1e-13)
    assert true <= 1e-12
    return x


@pytest.mark.parametrize("mode", [INTERIOR, EXTERIOR])
def test_densities_against_oracle_fp64_solve(mode):
    eps, K, N = 0.02, 128, 120
    pre = O.make_precompute(eps, mode, K, npan=8, nord=12, ntheta=40, tau=1e-10)
    c = L.uniform(N, eps, L.rng(1, 250 + mode))
    ref = _oracle_solution(pre, c)
    Is_ref, val_ref = S.outputs(pre.op.I, ref, N, mode)
    scale = np.abs(ref).max()
    ctx = ncs.Context(eps, mode, K, operator=(pre.idr.T, pre.idr.t_skel, pre.idr.th_skel, pre.op.I),
                      method=ncs.METHOD_DIRECT, tree_min_patches=100)
    ctx.set_patches(c)
    errs = {}
    for method in (ncs.METHOD_DIRECT, ncs.METHOD_TREE):
        ctx.set_method(method)
        for name, prec, tol in (("fp64", ncs.FP64, 1e-12), ("df64", ncs.DF64, 1e-12), ("mixed", ncs.MIXED, 1e-10)):
            r = ctx.solve(tol=tol, precision=prec)
            errs[(method, name)] = (np.abs(r["fhat"] - ref).max() / scale, abs(r["scalar"] - val_ref) / abs(val_ref))
    for k, (e, es) in errs.items():
        print(f"mode {mode} method {k[0]} {k[1]}: density error {e:.2e}, scalar error {es:.2e}")
    # direct products: the same compressed sums as the oracle
    assert errs[(ncs.METHOD_DIRECT, "fp64")][0] <= 1e-10
    assert errs[(ncs.METHOD_DIRECT, "df64")][0] <= 1e-10
    assert errs[(ncs.METHOD_DIRECT, "mixed")][0] <= 1e-6
    # the tree adds the incoming-grid interpolation (tolerance 1e-8)
    for name in ("fp64", "df64", "mixed"):
        assert errs[(ncs.METHOD_TREE, name)][0] <= 1e-6
        assert errs[(ncs.METHOD_TREE, name)][1] <= 1e-7
