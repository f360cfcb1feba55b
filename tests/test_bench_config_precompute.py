"""The library's own one-patch precompute at the settings of the 100 000-patch workload
(eps = 0.001, K = 136, 13 x 20 panels, default fine grid, ID tolerance 1e-11, the full
ladder of far-field representations) against the oracle at the same settings:
  * the radial profiles beta and I = w^T B (Sections 5 and 8, eq. getI) against the
    oracle's modal solver (brute theta quadrature of the full Green's function);
  * every representation of the ID ladder (Section 7.1, eq. Tmap) against the oracle's
    fine-grid far field (its own B and weights) at held-out targets beyond its radius.
Host path on CPU; the device path (collocation matrices, sketch, CPQR and T assembly on
the GPU) in the gpu-marked twin."""
import numpy as np
import pytest

from oracle import idcomp, onepatch
from oracle.kernels import EXTERIOR, INTERIOR, G_on_surface, chord
from paper_1906_04209_gb300 import ncs

EPS, K = 0.001, 136
_OP = {}


def _oracle(mode):
    if mode not in _OP:
        _OP[mode] = onepatch.solve_one_patch(EPS, mode, K, 13, 20, None)
    return _OP[mode]


def _check(ctx, mode):
    op = _oracle(mode)
    assert ctx.info()["nf"] == op.t_f.size
    tr, beta = ctx.onepatch()
    assert np.abs(tr - op.rad.t).max() <= 1e-15
    eb = np.abs(beta - op.beta).max() / np.abs(op.beta).max()
    eI = np.abs(ctx.operator()["I"] - op.I).max() / np.abs(op.I).max()
    assert eb <= 1e-10, eb
    assert eI <= 1e-10, eI
    xf = idcomp.fine_points(op)
    f = np.random.default_rng(7 + mode).standard_normal(K)
    src = op.w * (op.B @ f)
    rm, ps = ctx.reps()
    assert len(ps) >= 10 and rm[0] <= 2.0 * EPS * (1 + 1e-12)
    rng = np.random.default_rng(8 + mode)
    worst = 0.0
    for r in range(len(ps)):
        T, st, sth = ctx.rep(r)
        xt = idcomp.training_grid(EPS, 1e-11, nper=3, rho_min_factor=1.03 * rm[r] / EPS)
        xt = xt[rng.choice(len(xt), min(len(xt), 400), replace=False)]
        xs = np.stack([np.sin(st) * np.cos(sth), np.sin(st) * np.sin(sth), np.cos(st)], 1)
        ref = G_on_surface(chord(xt[:, None], xf[None]), mode) @ src
        lib = G_on_surface(chord(xt[:, None], xs[None]), mode) @ (T @ f)
        err = np.abs(lib - ref).max() / np.abs(ref).max()
        worst = max(worst, err)
        assert err < 1e-9, (r, rm[r], ps[r], err)
    return eb, eI, worst


@pytest.mark.parametrize("mode", [INTERIOR, EXTERIOR])
def test_host_precompute_at_workload_settings(libncs, mode):
    ctx = ncs.Context(EPS, mode, K, device_precompute=0)
    eb, eI, worst = _check(ctx, mode)
    print(f"mode {mode}: beta {eb:.1e}, I {eI:.1e}, worst ladder far field {worst:.1e}")


@pytest.mark.gpu
@pytest.mark.parametrize("mode", [INTERIOR, EXTERIOR])
def test_device_precompute_at_workload_settings(libncs, mode):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU test without a GPU"
    torch.cuda.set_device(0)
    ctx = ncs.Context(EPS, mode, K, device_precompute=1)
    t = ctx.timings()
    assert t[2] == 1.0 and t[6] == 1.0
    eb, eI, worst = _check(ctx, mode)
    print(f"mode {mode} (device): beta {eb:.1e}, I {eI:.1e}, worst ladder far field {worst:.1e}")
