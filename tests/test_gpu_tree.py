"""GPU parity of the tree product (Section 7, Step 3) against the oracle's
compressed sums (Section 7.1), element by element at sampled Zernike nodes, at
moderate N and at the full 100 000-patch workload size."""
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


def _ctx(pre, **kw):
    return ncs.Context(pre.eps, pre.mode, pre.K,
                       operator=(pre.idr.T, pre.idr.t_skel, pre.idr.th_skel, pre.op.I), **kw)


def _field(ctx, x, prec, N, Kstar):
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    zd = torch.empty(N * Kstar, dtype=torch.float64, device="cuda")
    ctx.field_dev(xd.data_ptr(), zd.data_ptr(), prec, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return zd.cpu().numpy().reshape(N, Kstar)


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_tree_vs_compressed_sums(small_pre, mode):
    eps = 0.01
    pre = small_pre(mode, eps=eps)
    N = 2500
    c = L.uniform(N, eps, L.rng(96))
    x = np.random.default_rng(11).standard_normal(N * pre.K)
    ctx = _ctx(pre, method=ncs.METHOD_TREE, grid_tol=1e-10)
    ctx.set_patches(c)
    st = ctx.tree_stats()
    assert st["grid_groups"] > 0 and st["levels"] >= 5
    patches = np.random.default_rng(12).choice(N, 12, replace=False)
    ref = O.id_field(pre, c, x, patches)
    scale = np.abs(ref).max()
    zf64 = _field(ctx, x, ncs.FP64, N, pre.Kstar)
    zfdf = _field(ctx, x, ncs.DF64, N, pre.Kstar)
    z64 = zf64[patches]
    n0 = ncs.launch_count()
    z32 = _field(ctx, x, ncs.FP32, N, pre.Kstar)[patches]
    n1 = ncs.launch_count()
    _field(ctx, x, ncs.FP32, N, pre.Kstar)
    # outgoing (pack + tensor-core GEMM), P2L, direct lists, L2P, plus one coefficient and
    # at most one L2L launch per level
    assert n1 - n0 == ncs.launch_count() - n1
    assert 5 + 1 <= n1 - n0 <= 5 + 2 * st["levels"]
    assert np.abs(z64 - ref).max() <= 1e-8 * scale
    # FP32 pair sums with the 3xTF32 outgoing map (a few 1e-6, see the direct parity test)
    assert np.abs(z32 - ref).max() <= 8e-6 * scale
    # float-float tree product = FP64 tree product to rounding (same grids, same lists)
    assert np.abs(zfdf - zf64).max() <= 1e-12 * np.abs(zf64).max()
    # the direct product on the same context agrees as well
    ctx.set_method(ncs.METHOD_DIRECT)
    zd = _field(ctx, x, ncs.FP64, N, pre.Kstar)[patches]
    assert np.abs(zd - ref).max() <= 1e-12 * scale


@pytest.mark.parametrize("layout", ["uniform", "vmf"])
def test_default_grid_tolerance(small_pre, layout):
    """At the default incoming-grid tolerance (1e-8) the tree product stays within 1e-8
    of the oracle's compressed sums (grid sizes from the trailing-coefficient rule)."""
    eps = 0.01
    pre = small_pre(INTERIOR, eps=eps)
    N = 4000
    c = L.uniform(N, eps, L.rng(99)) if layout == "uniform" else L.vmf_clusters(N, eps, L.rng(99))
    x = np.random.default_rng(19).standard_normal(N * pre.K)
    ctx = _ctx(pre, method=ncs.METHOD_TREE)
    ctx.set_patches(c)
    assert ctx.tree_stats()["grid_groups"] > 0
    patches = np.random.default_rng(20).choice(N, 12, replace=False)
    ref = O.id_field(pre, c, x, patches)
    z64 = _field(ctx, x, ncs.FP64, N, pre.Kstar)[patches]
    assert np.abs(z64 - ref).max() <= 1e-8 * np.abs(ref).max()


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_tree_solve_matches_direct(small_pre, mode):
    eps = 0.01
    pre = small_pre(mode, eps=eps)
    N = 2000
    c = L.jittered_fibonacci(N, eps, L.rng(97))
    ctx = _ctx(pre, method=ncs.METHOD_DIRECT)
    ctx.set_patches(c)
    # float-float products: FP64-accurate at a fraction of the FP64-pipe time
    rd = ctx.solve(tol=1e-10, precision=ncs.DF64)
    ctx.set_method(ncs.METHOD_TREE)
    rt = ctx.solve(tol=1e-10, precision=ncs.DF64)
    rm = ctx.solve(tol=1e-8, precision=ncs.MIXED)
    assert abs(rt["scalar"] - rd["scalar"]) <= 1e-8 * abs(rd["scalar"])
    assert np.abs(rt["fhat"] - rd["fhat"]).max() <= 1e-7 * np.abs(rd["fhat"]).max()
    assert rm["relres"] <= 1e-8
    assert np.abs(rm["fhat"] - rt["fhat"]).max() <= 1e-6 * np.abs(rt["fhat"]).max()


@pytest.mark.parametrize("update", [0, 1])
def test_mixed_solve_true_residual(small_pre, update):
    """The mixed solve's reported residual is the true one: b - A x recomputed with
    float-float products after the solve stays within the tolerance, with and without
    the FP32 residual update of the refinement."""
    eps = 0.01
    pre = small_pre(INTERIOR, eps=eps)
    N = 2500
    c = L.uniform(N, eps, L.rng(98))
    ctx = _ctx(pre, method=ncs.METHOD_TREE, grid_tol=1e-10, residual_update=update)
    ctx.set_patches(c)
    tol = 1e-9
    rm = ctx.solve(tol=tol, precision=ncs.MIXED)
    assert rm["relres"] <= tol
    b = np.tile(pre.P.sum(axis=1), N)
    xd = torch.tensor(rm["fhat"], dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    ctx.matvec_dev(xd.data_ptr(), yd.data_ptr(), ncs.DF64, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    true_rel = np.linalg.norm(b - yd.cpu().numpy()) / np.linalg.norm(b)
    assert true_rel <= 1.05 * tol
    assert abs(true_rel - rm["relres"]) <= 0.05 * tol


@pytest.mark.parametrize("layout,mode", [("fibonacci", INTERIOR), ("fibonacci", EXTERIOR), ("vmf", INTERIOR),
                                         ("vmf", EXTERIOR)])
def test_full_size_sampled(libncs, layout, mode):
    """The 100 000-patch workloads (eps = 0.001, K = 136; jittered Fibonacci and 20 vMF
    clusters; interior and exterior): tree product in the launch configuration the
    benchmark times, checked at 48 sampled (patch, node) outputs against the plain-C
    oracle sums."""
    c, eps, _, K = L.workload(3, layout=layout)
    pre = O.make_precompute(eps, mode, K, npan=8, nord=12, ntheta=40, tau=1e-10)
    N = len(c)
    ctx = _ctx(pre, method=ncs.METHOD_TREE)
    ctx.set_patches(c)
    x = np.random.default_rng(13).standard_normal(N * K)
    rng = np.random.default_rng(14)
    patches = rng.choice(N, 48)
    nodes = rng.choice(pre.Kstar, 48)
    ref = native.rows(pre, c, x, patches, nodes)
    scale = np.abs(ref).max()
    zdf = _field(ctx, x, ncs.DF64, N, pre.Kstar)[patches, nodes]
    z32 = _field(ctx, x, ncs.FP32, N, pre.Kstar)[patches, nodes]
    edf, e32 = np.abs(zdf - ref).max() / scale, np.abs(z32 - ref).max() / scale
    print(f"N=1e5 {layout} mode {mode}: float-float error {edf:.2e}, FP32 error {e32:.2e}")
    # float-float: only the incoming-grid interpolation separates the tree from the sums
    assert edf <= 1e-8
    assert e32 <= 1e-5


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_multilevel_representations(mode):
    """Several outgoing representations (far fields beyond 2, 3, 4, 6, 8 eps), each an
    oracle ID: the tree and the direct product pick per interaction the coarsest valid
    one and still match the single-representation compressed sums."""
    from oracle import idcomp, onepatch, zernike
    eps, K = 0.01, 10
    op = onepatch.solve_one_patch(eps, mode, K, 6, 10, 24)
    radii = [2.0, 3.0, 4.0, 6.0, 8.0]
    reps = []
    for r in radii:
        idr = idcomp.interpolative_decomposition(op, 1e-11, rho_min_factor=r)
        reps.append((idr.T, idr.t_skel, idr.th_skel))
    P, rz, thz = zernike.transform(K)
    pre = O.Precompute(eps, mode, K, op, idcomp.interpolative_decomposition(op, 1e-11), P, rz, thz)
    N = 1500
    c = L.uniform(N, eps, L.rng(98))
    x = np.random.default_rng(15).standard_normal(N * K)
    ctx = ncs.Context(eps, mode, K, operator=dict(rho_min=np.array(radii) * eps, reps=reps, I=op.I),
                      method=ncs.METHOD_TREE, grid_tol=1e-10)
    ctx.set_patches(c)
    rm, ps = ctx.reps()
    assert len(ps) == 5 and ps[0] > ps[-1]
    patches = np.random.default_rng(16).choice(N, 8, replace=False)
    ref = O.id_field(pre, c, x, patches)
    scale = np.abs(ref).max()
    zt = _field(ctx, x, ncs.FP64, N, pre.Kstar)[patches]
    ctx.set_method(ncs.METHOD_DIRECT)
    zd = _field(ctx, x, ncs.FP64, N, pre.Kstar)[patches]
    assert np.abs(zd - ref).max() <= 1e-9 * scale
    assert np.abs(zt - ref).max() <= 1e-8 * scale
