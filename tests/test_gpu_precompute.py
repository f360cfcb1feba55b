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


@pytest.mark.parametrize("eps,mode,K,kw", [
    (0.001, INTERIOR, 136, {}),                           # the N = 1e5 workload's patch
    (0.05, EXTERIOR, 64, {}),                             # the N = 10 workload's patch
    (0.02, EXTERIOR, 171, dict(npan=8, nord=12)),         # 18 modes: the 32-mode kernel
    (0.03, INTERIOR, 21, dict(npan=6, nord=32)),          # the largest panel order on the device
])
def test_device_collocation_matches_host(eps, mode, K, kw):
    """The modal collocation matrices (Section 8.2) formed on the device give the same
    one-patch solution as the host loop: same quadrature rules and theta rule, so the radial
    profiles beta and I = w^T B agree to rounding amplified by the collocation system."""
    kw = dict(kw, ntheta_fine=40, method=ncs.METHOD_DIRECT, id_ladder_max=0.0)
    dev = ncs.Context(eps, mode, K, device_precompute=1, **kw)
    host = ncs.Context(eps, mode, K, device_precompute=0, **kw)
    td, th = dev.timings(), host.timings()
    assert td[6] == 1.0 and th[6] == 0.0
    trd, bd = dev.onepatch()
    trh, bh = host.onepatch()
    assert np.array_equal(trd, trh)
    err = np.abs(bd - bh).max() / np.abs(bh).max()
    Id, Ih = dev.operator()["I"], host.operator()["I"]
    errI = np.abs(Id - Ih).max() / np.abs(Ih).max()
    print(f"eps {eps} mode {mode} K {K}: beta rel diff {err:.1e}, I rel diff {errI:.1e}; collocation "
          f"{td[7]:.3f} s (device) vs {th[7]:.3f} s (host), one-patch {td[0]:.3f} vs {th[0]:.3f} s")
    assert err <= 1e-10, err
    assert errI <= 1e-12, errI


def test_device_collocation_beyond_kernel_limits_uses_host():
    # panel order 33 exceeds the device kernel's limit: the host loop forms the matrices
    c = ncs.Context(0.05, EXTERIOR, 10, npan=4, nord=33, ntheta_fine=24, method=ncs.METHOD_DIRECT,
                    id_ladder_max=0.0, device_precompute=1)
    assert c.timings()[6] == 0.0


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_device_onepatch_matches_oracle(mode):
    """The one-patch solution with its collocation matrices formed on the device against the
    oracle's modal solver (brute quadrature of the full Green's function in theta, scipy
    rules): the same bar as the host path's CPU test."""
    from oracle import onepatch
    eps, K, npan, nord, nth = 0.05, 21, 7, 12, 30
    c = ncs.Context(eps, mode, K, npan=npan, nord=nord, ntheta_fine=nth, device_precompute=1,
                    method=ncs.METHOD_DIRECT)
    assert c.timings()[6] == 1.0
    tr, beta = c.onepatch()
    op = onepatch.solve_one_patch(eps, mode, K, npan, nord, nth)
    assert np.abs(tr - op.rad.t).max() < 1e-15
    assert np.abs(beta - op.beta).max() < 1e-11 * np.abs(op.beta).max()
    assert np.abs(c.operator()["I"] - op.I).max() < 1e-11 * np.abs(op.I).max()
