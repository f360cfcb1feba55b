"""The interpolative decompositions of the one-patch precompute (Section 7.1) run on the
device (sketch, column-pivoted QRs, T assembly) give the same compressed operator as the
host path: same skeleton counts (within one point), and products that agree to the ID
tolerance."""
import time

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


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_device_sketch_matches_host(mode):
    eps, K = 0.02, 21
    kw = dict(npan=8, nord=12, ntheta_fine=40, method=ncs.METHOD_DIRECT)
    t0 = time.time()
    dev = ncs.Context(eps, mode, K, device_precompute=1, **kw)
    t_dev = time.time() - t0
    t0 = time.time()
    host = ncs.Context(eps, mode, K, device_precompute=0, **kw)
    t_host = time.time() - t0
    assert dev.timings()[2] == 1.0 and host.timings()[2] == 0.0
    rd, pd = dev.reps()
    rh, ph = host.reps()
    assert np.array_equal(rd, rh)
    assert np.all(np.abs(np.asarray(pd) - np.asarray(ph)) <= 1)
    N = 200
    c = L.uniform(N, eps, L.rng(60 + mode))
    x = np.random.default_rng(61).standard_normal(N * K)
    ys = []
    for ctx in (dev, host):
        ctx.set_patches(c)
        ys.append(ctx.matvec(x, ncs.FP64))
    scale = np.abs(ys[1] - x).max()
    assert np.abs(ys[0] - ys[1]).max() <= 1e-9 * scale
    print(f"mode {mode}: precompute {t_dev:.2f} s (device sketch) vs {t_host:.2f} s (host), p {pd[0]} / {ph[0]}")
