"""GPU parity at the sizes of the smaller named workloads (Section 9 set-ups):
  * exterior N = 10, eps = 0.05, K = 64: dense oracle solve (eq. opinteqnsdisc, LU);
  * interior N = 1000, eps = 0.02, K = 128: direct and tree products against the oracle's
    compressed sums (Section 7.1), FP64 GMRES to 1e-10 with both;
  * exterior N = 1e4, eps = 0.005, K = 136: mixed precision against the FP64-accurate
    (float-float) path and the oracle's sums; the density error is reported.
The library takes the oracle's ID (T, skeleton, I) through ncs_create_from_operator so
both sides sum the same compressed operator; one case also uses the library's own
precompute."""
import numpy as np
import pytest

from oracle import native, operator as O, solve as S
from paper_1906_04209_gb300 import layouts as L, ncs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda(libncs):
    assert torch.cuda.is_available(), "GPU test without a GPU"
    torch.cuda.set_device(0)


def _ctx(pre, **kw):
    return ncs.Context(pre.eps, pre.mode, pre.K,
                       operator=(pre.idr.T, pre.idr.t_skel, pre.idr.th_skel, pre.op.I), **kw)


def _field(ctx, x, prec, N, Kstar):
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    zd = torch.empty(N * Kstar, dtype=torch.float64, device="cuda")
    ctx.field_dev(xd.data_ptr(), zd.data_ptr(), prec, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return zd.cpu().numpy().reshape(N, Kstar)


def test_exterior_N10_K64_dense():
    c, eps, mode, K = L.workload(0)
    pre = O.make_precompute(eps, mode, K)
    N = len(c)
    f_ref = S.dense_solve(O.dense_operator(pre, c), O.rhs(pre, N))
    Is_ref, C_ref = S.outputs(pre.op.I, f_ref, N, mode)
    ctx = _ctx(pre, method=ncs.METHOD_DIRECT)
    ctx.set_patches(c)
    r = ctx.solve(tol=1e-12, precision=ncs.FP64)
    print(f"N=10 K=64 exterior: C = {r['scalar']:.12f} (oracle {C_ref:.12f}), {r['iterations']} iterations")
    assert abs(r["scalar"] - C_ref) <= 1e-9 * C_ref
    assert abs(r["Isigma"] - Is_ref) <= 1e-9 * Is_ref
    assert np.abs(r["fhat"] - f_ref).max() <= 1e-9 * np.abs(f_ref).max()
    rm = ctx.solve(tol=1e-10, precision=ncs.MIXED)
    assert abs(rm["scalar"] - C_ref) <= 1e-9 * C_ref
    # the library's own precompute (its own one-patch solve and ID) agrees as well
    own = ncs.Context(eps, mode, K, method=ncs.METHOD_DIRECT)
    own.set_patches(c)
    ro = own.solve(tol=1e-12, precision=ncs.FP64)
    assert abs(ro["scalar"] - C_ref) <= 1e-9 * C_ref


def test_interior_N1000_K128():
    c, eps, mode, K = L.workload(1)
    pre = O.make_precompute(eps, mode, K, npan=8, nord=12, ntheta=40, tau=1e-10)
    N = len(c)
    x = np.random.default_rng(31).standard_normal(N * K)
    rng = np.random.default_rng(32)
    patches, nodes = rng.choice(N, 64), rng.choice(pre.Kstar, 64)
    ref = native.rows(pre, c, x, patches, nodes)
    scale = np.abs(ref).max()
    ctx = _ctx(pre, method=ncs.METHOD_DIRECT)
    ctx.set_patches(c)
    zd = _field(ctx, x, ncs.FP64, N, pre.Kstar)[patches, nodes]
    assert np.abs(zd - ref).max() <= 1e-12 * scale
    rd = ctx.solve(tol=1e-10, precision=ncs.DF64, want_fhat=False)
    ctx.set_method(ncs.METHOD_TREE)
    zt = _field(ctx, x, ncs.FP64, N, pre.Kstar)[patches, nodes]
    z32 = _field(ctx, x, ncs.FP32, N, pre.Kstar)[patches, nodes]
    assert np.abs(zt - ref).max() <= 1e-7 * scale
    assert np.abs(z32 - ref).max() <= 1e-5 * scale
    rt = ctx.solve(tol=1e-10, precision=ncs.FP64, want_fhat=False)
    print(f"N=1000 K=128 interior: mu direct {rd['scalar']:.12f}, tree {rt['scalar']:.12f}, "
          f"{rt['iterations']} iterations")
    assert rd["relres"] <= 1e-10 and rt["relres"] <= 1e-10
    assert abs(rt["scalar"] - rd["scalar"]) <= 1e-8 * abs(rd["scalar"])


def test_exterior_N1e4_K136_mixed():
    c, eps, mode, K = L.workload(2)
    pre = O.make_precompute(eps, mode, K, npan=8, nord=12, ntheta=40, tau=1e-10)
    N = len(c)
    x = np.random.default_rng(33).standard_normal(N * K)
    rng = np.random.default_rng(34)
    patches, nodes = rng.choice(N, 48), rng.choice(pre.Kstar, 48)
    ref = native.rows(pre, c, x, patches, nodes)
    scale = np.abs(ref).max()
    ctx = _ctx(pre, method=ncs.METHOD_TREE)
    ctx.set_patches(c)
    zdf = _field(ctx, x, ncs.DF64, N, pre.Kstar)[patches, nodes]
    z32 = _field(ctx, x, ncs.FP32, N, pre.Kstar)[patches, nodes]
    assert np.abs(zdf - ref).max() <= 1e-7 * scale
    assert np.abs(z32 - ref).max() <= 1e-5 * scale
    # both solved to 1e-10, so that the density difference measures precision, not the
    # GMRES tolerance (two iterates with residual 1e-8 may differ by cond(A) * 1e-8)
    rdf = ctx.solve(tol=1e-10, precision=ncs.DF64)
    rm = ctx.solve(tol=1e-10, precision=ncs.MIXED)
    err = np.abs(rm["fhat"] - rdf["fhat"]).max() / np.abs(rdf["fhat"]).max()
    print(f"N=1e4 K=136 exterior: C mixed {rm['scalar']:.12f}, float-float {rdf['scalar']:.12f}, "
          f"density error {err:.2e}")
    assert rm["relres"] <= 1e-10 and rdf["relres"] <= 1e-10
    assert err <= 1e-6
    assert abs(rm["scalar"] - rdf["scalar"]) <= 1e-8 * abs(rdf["scalar"])
