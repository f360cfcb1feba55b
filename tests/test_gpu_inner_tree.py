"""The mixed solve's inner tree (inner_grid_tol, layouts of 10 000 patches and more): the inner
FP32 solves and the FP32 residual update run on incoming grids to a looser tolerance (fewer
grid points and pair evaluations), the float-float refinement residuals on the product's grids
(grid_tol). The converged solution is that of the product's operator: the same mean first
passage time and capacitance as with one tree throughout, both to the requested true residual."""
import numpy as np
import pytest

from oracle.kernels import EXTERIOR, INTERIOR
from paper_1906_04209_gb300 import layouts as L, ncs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda(libncs):
    assert torch.cuda.is_available(), "GPU test without a GPU"
    torch.cuda.set_device(0)


@pytest.mark.parametrize("mode", [INTERIOR, EXTERIOR])
def test_inner_tree_solve_matches_single_tree(mode):
    eps, K, N = 0.002, 21, 12000
    c = L.jittered_fibonacci(N, eps, L.rng(95, mode))
    kw = dict(npan=6, nord=10, ntheta_fine=24, method=ncs.METHOD_TREE)
    out = {}
    for itol in (1e-5, 0.0):
        ctx = ncs.Context(eps, mode, K, inner_grid_tol=itol, **kw)
        ctx.set_patches(c)
        r = ctx.solve(tol=1e-10, precision=ncs.MIXED)
        out[itol] = (r, ctx.info(), ctx.solve_stats())
    (ra, ia, sa), (rb, ib, sb) = out[1e-5], out[0.0]
    print(f"mode {mode}: grid points {ia['grid_points']} / inner {ia['inner_grid_points']}, pairs "
          f"{ia['tree_pairs']} / inner {ia['inner_tree_pairs']}; iterations {ra['iterations']} vs {rb['iterations']}, "
          f"scalar {ra['scalar']:.12f} vs {rb['scalar']:.12f}")
    assert 0 < ia["inner_grid_points"] < ia["grid_points"]
    assert 0 < ia["inner_tree_pairs"] < ia["tree_pairs"]
    assert ib["inner_grid_points"] == 0 and ib["inner_tree_pairs"] == 0
    assert ra["relres"] <= 1e-10 and rb["relres"] <= 1e-10
    assert sa["recomputed"] == 1.0 and sb["recomputed"] == 1.0
    assert abs(ra["scalar"] - rb["scalar"]) <= 1e-9 * abs(rb["scalar"])


def test_no_inner_tree_below_threshold():
    c = L.jittered_fibonacci(3000, 0.004, L.rng(97))
    ctx = ncs.Context(0.004, INTERIOR, 21, npan=6, nord=10, ntheta_fine=24, method=ncs.METHOD_TREE)
    ctx.set_patches(c)
    r = ctx.solve(tol=1e-10, precision=ncs.MIXED)
    assert r["relres"] <= 1e-10
    assert ctx.info()["inner_grid_points"] == 0
