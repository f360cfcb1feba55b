"""The tree product's autotuner (ncs_tune): on a 20 000-patch layout of the benchmark's
family (eps = 0.001, K = 136, jittered Fibonacci, the library's own precompute) it times
the pair-kernel variants and the tree knobs, keeps only configurations whose FP32 product
matches the float-float product, and the chosen one is no slower than the default; a
second context of the same workload takes the choice from the cache file without trials;
the mixed solve under the tuned configuration gives the same answer."""
import numpy as np
import pytest

from oracle.kernels import INTERIOR
from paper_1906_04209_gb300 import layouts as L, ncs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda(libncs):
    assert torch.cuda.is_available(), "GPU test without a GPU"
    torch.cuda.set_device(0)


def _field(ctx, x, prec, N, Kstar):
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    zd = torch.empty(N * Kstar, dtype=torch.float64, device="cuda")
    ctx.field_dev(xd.data_ptr(), zd.data_ptr(), prec, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return zd.cpu().numpy()


def test_tune_chooses_accurate_faster_configuration(tmp_path):
    c, eps, mode, K = L.workload(3, N=20000)
    cache = str(tmp_path / "tune.txt")
    ctx = ncs.Context(eps, mode, K, method=ncs.METHOD_TREE)
    ctx.set_patches(c)
    r0 = ctx.solve(tol=1e-9, precision=ncs.MIXED, want_fhat=False)
    cfg, rep = ctx.tune(flags=3, cache_path=cache)
    print(f"tuned {cfg}: {rep}")
    assert rep["from_cache"] == 0.0 and rep["trial_products"] > 10
    assert rep["error"] <= 2e-5
    assert rep["tuned_ms"] <= 1.03 * rep["default_ms"]
    assert ctx.get_tuning() == cfg
    Kstar = ctx.info()["Kstar"]
    x = np.random.default_rng(3).standard_normal(len(c) * K)
    z32 = _field(ctx, x, ncs.FP32, len(c), Kstar)
    zdf = _field(ctx, x, ncs.DF64, len(c), Kstar)
    assert np.abs(z32 - zdf).max() <= 2e-5 * np.abs(zdf).max()
    r1 = ctx.solve(tol=1e-9, precision=ncs.MIXED, want_fhat=False)
    assert r1["relres"] <= 1e-9
    assert abs(r1["scalar"] - r0["scalar"]) <= 1e-9 * abs(r0["scalar"])
    # a second context of the same workload reads the choice from the cache
    ctx2 = ncs.Context(eps, mode, K, method=ncs.METHOD_TREE)
    ctx2.set_patches(c)
    cfg2, rep2 = ctx2.tune(flags=3, cache_path=cache)
    assert rep2["from_cache"] == 1.0 and rep2["trial_products"] == 0.0
    assert cfg2 == cfg


def test_tune_errors():
    c, eps, mode, K = L.workload(3, N=3000)
    ctx = ncs.Context(eps, mode, K, method=ncs.METHOD_DIRECT, npan=8, nord=12, ntheta_fine=40)
    ctx.set_patches(c)
    with pytest.raises(ncs.NcsError) as e:
        ctx.tune(flags=3)
    assert e.value.code == ncs.NCS_E_STATE
    with pytest.raises(ncs.NcsError) as e:
        ctx.tune(flags=0)
    assert e.value.code == ncs.NCS_E_INPUT
