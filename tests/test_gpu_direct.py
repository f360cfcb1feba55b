"""GPU parity of the direct (no tree) product and the solve against the oracle.
All calls go through the C ABI (libncs.so) via the ctypes binding."""
import numpy as np
import pytest

from oracle import operator as O, solve as S
from oracle.kernels import EXTERIOR, INTERIOR, G_off_surface
from paper_1906_04209_gb300 import layouts as L, ncs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda(libncs):
    assert torch.cuda.is_available(), "GPU test without a GPU"
    torch.cuda.set_device(0)


def _ctx_from_oracle(pre, **kw):
    return ncs.Context(pre.eps, pre.mode, pre.K,
                       operator=(pre.idr.T, pre.idr.t_skel, pre.idr.th_skel, pre.op.I), **kw)


def _field_gpu(ctx, x, prec, N, Kstar):
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    zd = torch.empty(N * Kstar, dtype=torch.float64, device="cuda")
    ctx.field_dev(xd.data_ptr(), zd.data_ptr(), prec, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return zd.cpu().numpy().reshape(N, Kstar)


# FP32 field tolerance relative to max |z|: SIMT outgoing map ~FP32 rounding; the 3xTF32
# tensor-core map splits each operand into TF32 hi + lo (2^-22 relative per operand), so
# its coefficients, and the field, carry a few times more error.
FP32_TOL = {0: 2e-6, 1: 6e-6}


@pytest.mark.parametrize("tc", [0, 1])
@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
@pytest.mark.parametrize("N", [1, 2, 9, 37])
def test_field_parity_shared_operator(small_pre, mode, N, tc):
    """Same operator data on both sides: GPU z vs oracle compressed sums, element by
    element. N = 9 and 37 leave ragged source tiles (8 patches per tile)."""
    pre = small_pre(mode)
    c = L.uniform(N, 0.1, L.rng(91, N))
    x = np.random.default_rng(N).standard_normal(N * pre.K)
    ctx = _ctx_from_oracle(pre, method=ncs.METHOD_DIRECT, tensor_cores=tc)
    ctx.set_patches(c)
    ref = O.id_field(pre, c, x)
    scale = max(np.abs(ref).max(), 1e-300)
    z64 = _field_gpu(ctx, x, ncs.FP64, N, pre.Kstar)
    z32 = _field_gpu(ctx, x, ncs.FP32, N, pre.Kstar)
    zdf = _field_gpu(ctx, x, ncs.DF64, N, pre.Kstar)
    if N == 1:
        assert np.abs(z64).max() == 0.0 and np.abs(z32).max() == 0.0 and np.abs(zdf).max() == 0.0
        return
    assert np.abs(z64 - ref).max() <= 1e-12 * scale
    assert np.abs(zdf - ref).max() <= 1e-12 * scale
    assert np.abs(z32 - ref).max() <= FP32_TOL[tc] * scale


def test_context_precision(small_pre):
    """Calls given PRECISION_DEFAULT run at the context precision (ncs_set_precision):
    a solve at the default (mixed) equals the explicit mixed solve, products at MIXED run
    in FP32, and after set_precision(DF64) both run in float-float."""
    pre = small_pre(INTERIOR)
    N = 10
    c = L.uniform(N, 0.1, L.rng(95))
    ctx = _ctx_from_oracle(pre, method=ncs.METHOD_DIRECT)
    ctx.set_patches(c)
    x = np.random.default_rng(3).standard_normal(N * pre.K)
    assert np.array_equal(ctx.matvec(x, ncs.PRECISION_DEFAULT), ctx.matvec(x, ncs.FP32))
    r0 = ctx.solve(tol=1e-10, precision=ncs.PRECISION_DEFAULT)
    r1 = ctx.solve(tol=1e-10, precision=ncs.MIXED)
    assert r0["scalar"] == r1["scalar"] and r0["iterations"] == r1["iterations"]
    ctx.set_precision(ncs.DF64)
    assert np.array_equal(ctx.matvec(x, ncs.PRECISION_DEFAULT), ctx.matvec(x, ncs.DF64))
    r2 = ctx.solve(tol=1e-10, precision=ncs.PRECISION_DEFAULT)
    r3 = ctx.solve(tol=1e-10, precision=ncs.DF64)
    assert r2["scalar"] == r3["scalar"]


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_matvec_host_and_device_agree(small_pre, mode):
    pre = small_pre(mode)
    N = 12
    c = L.uniform(N, 0.1, L.rng(92))
    x = np.random.default_rng(7).standard_normal(N * pre.K)
    ctx = _ctx_from_oracle(pre, method=ncs.METHOD_DIRECT)
    ctx.set_patches(c)
    y = ctx.matvec(x, ncs.FP64)
    ref = O.id_matvec(pre, c, x)
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    ctx.matvec_dev(xd.data_ptr(), yd.data_ptr(), ncs.FP64, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert np.array_equal(yd.cpu().numpy(), y)


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_library_precompute_end_to_end(small_pre, mode):
    """The library's own precompute + GPU product vs the oracle's dense operator of
    eq. opinteqnsdisc (no compression on the oracle side): agreement to the ID level."""
    pre = small_pre(mode, ntheta=44)
    N = 7
    c = L.uniform(N, 0.1, L.rng(93))
    x = np.random.default_rng(8).standard_normal(N * pre.K)
    ctx = ncs.Context(0.1, mode, pre.K, npan=6, nord=10, ntheta_fine=44, method=ncs.METHOD_DIRECT)
    ctx.set_patches(c)
    y = ctx.matvec(x, ncs.FP64)
    ref = O.fine_matvec(pre, c, x)
    assert np.abs(y - ref).max() <= 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_solve_vs_oracle(small_pre, mode):
    pre = small_pre(mode)
    N = 8
    c = L.uniform(N, 0.1, L.rng(94))
    ctx = _ctx_from_oracle(pre, method=ncs.METHOD_DIRECT)
    ctx.set_patches(c)
    b = O.rhs(pre, N)
    x_ref, it_ref, _, _ = S.gmres(lambda v: O.id_matvec(pre, c, v), b, 1e-13)
    Is_ref, val_ref = S.outputs(pre.op.I, x_ref, N, mode)
    r = ctx.solve(tol=1e-12, precision=ncs.FP64)
    assert r["relres"] <= 1e-11
    assert np.abs(r["fhat"] - x_ref).max() <= 1e-10 * np.abs(x_ref).max()
    assert abs(r["scalar"] - val_ref) <= 1e-10 * abs(val_ref)
    assert abs(r["Isigma"] - Is_ref) <= 1e-10 * abs(Is_ref)
    rm = ctx.solve(tol=1e-10, precision=ncs.MIXED)
    assert rm["relres"] <= 1e-10
    assert np.abs(rm["fhat"] - x_ref).max() <= 1e-8 * np.abs(x_ref).max()
    rd = ctx.solve(tol=1e-11, precision=ncs.DF64)
    assert np.abs(rd["fhat"] - x_ref).max() <= 1e-9 * np.abs(x_ref).max()
    r32 = ctx.solve(tol=1e-5, precision=ncs.FP32)
    assert np.abs(r32["fhat"] - x_ref).max() <= 1e-4 * np.abs(x_ref).max()


def test_single_patch_solve(small_pre):
    pre = small_pre(INTERIOR)
    ctx = _ctx_from_oracle(pre, method=ncs.METHOD_DIRECT)
    ctx.set_patches([[0.0, 0.0, 1.0]])
    r = ctx.solve(tol=1e-12, precision=ncs.FP64)
    b = O.rhs(pre, 1)
    assert np.abs(r["fhat"] - b).max() <= 1e-14
    Is, mu = S.outputs(pre.op.I, b, 1, INTERIOR)
    assert abs(r["scalar"] - mu) <= 1e-13 * mu


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_eval_far_targets(small_pre, mode):
    """Single-layer potential off the patches (eqs. urep / intBVPansatz with the
    off-surface Green's functions), transformed to ubar / vbar."""
    pre = small_pre(mode)
    N = 5
    c = L.uniform(N, 0.1, L.rng(95))
    ctx = _ctx_from_oracle(pre, method=ncs.METHOD_DIRECT)
    ctx.set_patches(c)
    fhat = np.random.default_rng(9).standard_normal(N * pre.K)
    r = 2.0 if mode == EXTERIOR else 0.5
    tg = []
    rng = np.random.default_rng(10)
    while len(tg) < 16:
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        if np.arccos(np.clip(c @ v, -1, 1)).min() > 3 * pre.eps:
            tg.append(r * v)
    tg = np.array(tg)
    out = ctx.eval(tg, fhat)
    rho = O.outgoing(pre, fhat, N)
    src = O.skeleton_points_all(pre, c).reshape(-1, 3)
    u = np.array([np.sum(G_off_surface(t[None, :], src, mode) * rho.ravel()) for t in tg])
    Is, _ = S.outputs(pre.op.I, fhat, N, mode)
    ref = 1 - u if mode == EXTERIOR else (u - 1) / (3 * (-Is)) + (1 - r * r) / 6
    assert np.abs(out - ref).max() <= 1e-11 * np.abs(ref).max()
