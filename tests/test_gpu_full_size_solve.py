"""The metric's solve at full size: the 100 000-patch workload (eps = 0.001, K = 136,
13.6 M unknowns, the library's own precompute and tree, the launch configuration the
benchmark times), solved to a 1e-10 relative residual in mixed precision and with
float-float products (FP64-accurate, Section 7 Step 3). The float-float product itself is
pinned to the oracle's compressed sums at sampled outputs at this size (test_gpu_tree);
here the two solutions must agree (density <= 1e-6 relative, mu to 1e-8), and each
solution's true residual b - A x, recomputed after the solve with a float-float product,
must meet the tolerance."""
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


def _true_residual(ctx, fhat, b):
    xd = torch.tensor(fhat, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    ctx.matvec_dev(xd.data_ptr(), yd.data_ptr(), ncs.DF64, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return float(torch.linalg.norm(b - yd) / torch.linalg.norm(b))


@pytest.mark.parametrize("layout,mode", [("fibonacci", INTERIOR), ("vmf", EXTERIOR)])
def test_full_size_mixed_vs_float_float(layout, mode):
    c, eps, _, K = L.workload(3, layout=layout)
    N = len(c)
    ctx = ncs.Context(eps, mode, K, method=ncs.METHOD_TREE)
    ctx.set_patches(c)
    P = ctx.operator()["P"]
    b = torch.tensor(np.tile(P.sum(axis=1), N), dtype=torch.float64, device="cuda")
    tol = 1e-10
    rdf = ctx.solve(tol=tol, precision=ncs.DF64)
    rm = ctx.solve(tol=tol, precision=ncs.MIXED)
    st = ctx.solve_stats()
    tdf, tm = _true_residual(ctx, rdf["fhat"], b), _true_residual(ctx, rm["fhat"], b)
    err = np.abs(rm["fhat"] - rdf["fhat"]).max() / np.abs(rdf["fhat"]).max()
    emu = abs(rm["scalar"] - rdf["scalar"]) / abs(rdf["scalar"])
    print(f"N=1e5 {layout} mode {mode}: scalar mixed {rm['scalar']:.12f}, float-float {rdf['scalar']:.12f} "
          f"(rel {emu:.1e}); density error {err:.2e}; true residuals {tm:.2e} / {tdf:.2e}; "
          f"mixed {rm['iterations']} products ({st['gmres_steps']:.0f} FP32 steps, "
          f"{st['residual_products']:.0f} float-float residuals), float-float {rdf['iterations']}")
    assert rdf["relres"] <= tol and rm["relres"] <= tol
    assert tdf <= 1.05 * tol and tm <= 1.05 * tol
    assert err <= 1e-6
    assert emu <= 1e-8
