"""Batched solve of independent spheres (uneven N and eps, both modes) through the C ABI:
every instance matches its own single-context solve."""
import numpy as np
import pytest

from oracle import operator as O, solve as S
from paper_1906_04209_gb300 import layouts as L, ncs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda(libncs):
    assert torch.cuda.is_available(), "GPU test without a GPU"
    torch.cuda.set_device(0)


def test_batch_matches_individual():
    g = L.rng(77)
    inst = []
    for b in range(6):
        N = int(g.integers(20, 300))
        eps = float(g.uniform(0.01, 0.02))
        inst.append((L.uniform(N, eps, L.rng(77, b + 1)), eps, b % 2))
    kw = dict(npan=6, nord=10, ntheta_fine=24, method=ncs.METHOD_DIRECT)
    out = ncs.batch_solve(inst, 21, tol=1e-10, precision=ncs.MIXED, workers=3, **kw)
    assert out["rc"] == 0 and (out["status"] == 0).all()
    assert out["seconds"][2] > 0
    for b, (c, eps, mode) in enumerate(inst):
        ctx = ncs.Context(eps, mode, 21, **kw)
        ctx.set_patches(c)
        r = ctx.solve(tol=1e-10, precision=ncs.MIXED)
        assert abs(out["scalar"][b] - r["scalar"]) <= 1e-9 * abs(r["scalar"])
        assert out["relres"][b] <= 1e-10


def test_batch_vs_oracle():
    """Batched mixed-precision solves of uneven spheres (both modes, distinct eps)
    against the oracle's dense solve of the uncompressed system (eq. opinteqnsdisc)."""
    g = L.rng(78)
    inst = []
    for b, N in enumerate((8, 15, 24, 40)):
        eps = float(g.uniform(0.03, 0.06))
        inst.append((L.uniform(N, eps, L.rng(78, b + 1)), eps, b % 2))
    K, kw = 21, dict(npan=6, nord=10, ntheta_fine=24, method=ncs.METHOD_DIRECT)
    out = ncs.batch_solve(inst, K, tol=1e-10, precision=ncs.MIXED, workers=2, **kw)
    assert out["rc"] == 0 and (out["status"] == 0).all()
    for b, (c, eps, mode) in enumerate(inst):
        pre = O.make_precompute(eps, mode, K, npan=6, nord=10, ntheta=24, with_id=False)
        N = len(c)
        fhat = S.dense_solve(O.dense_operator(pre, c), O.rhs(pre, N))
        Is, val = S.outputs(pre.op.I, fhat, N, mode)
        assert abs(out["scalar"][b] - val) <= 1e-8 * abs(val)
        assert abs(out["Isigma"][b] - Is) <= 1e-8 * abs(Is)


def test_block_dots():
    """The Arnoldi projections V^T w through the C ABI against numpy."""
    rng = np.random.default_rng(5)
    n, k = 100_003, 37
    V = rng.standard_normal((k, n))
    w = rng.standard_normal(n)
    Vd = torch.tensor(V, device="cuda")
    wd = torch.tensor(w, device="cuda")
    out = torch.empty(k, dtype=torch.float64, device="cuda")
    ncs.block_dots(n, k, Vd.data_ptr(), n, wd.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    ref = V @ w
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12 * np.abs(V).max() * np.abs(w).max() * np.sqrt(n)


def test_batch_workload_small_instances_vs_oracle():
    """The 256-sphere batch workload (K = 128, uneven N and eps, both modes): every instance
    with at most 60 patches (9 of them), solved by ncs_batch_solve with the library's own
    precompute at reduced panels, against the oracle's GMRES on its own compressed
    operator at the same settings (plain-C sums at every Zernike node)."""
    from oracle import native
    work = L.batch_workload(256)
    sel = [(c, e, m) for c, e, m, _ in work if len(c) <= 60]
    assert len(sel) == 9
    K, kw = 128, dict(npan=8, nord=12, ntheta_fine=40, method=ncs.METHOD_DIRECT)
    out = ncs.batch_solve(sel, K, tol=1e-10, precision=ncs.MIXED, workers=4, **kw)
    assert out["rc"] == 0 and (out["status"] == 0).all()
    for b, (c, eps, mode) in enumerate(sel):
        pre = O.make_precompute(eps, mode, K, npan=8, nord=12, ntheta=40, tau=1e-11)
        N = len(c)
        pt, nd = np.repeat(np.arange(N), pre.Kstar), np.tile(np.arange(pre.Kstar), N)

        def matvec(x):
            return x + (native.rows(pre, c, x, pt, nd).reshape(N, pre.Kstar) @ pre.P.T).ravel()

        x, _, _, true = S.gmres(matvec, O.rhs(pre, N), 1e-12)
        Is, val = S.outputs(pre.op.I, x, N, mode)
        print(f"instance N={N} eps={eps:.4f} mode {mode}: library {out['scalar'][b]:.12f}, oracle {val:.12f}")
        assert abs(out["scalar"][b] - val) <= 1e-8 * abs(val)
        assert out["relres"][b] <= 1e-10


def test_grouped_small_spheres_match_separate_contexts():
    """Spheres below the tree threshold solved as one grouped system (batch_grouped = 1:
    concatenated patches, per-instance operators and GMRES states) against the same batch
    solved on one context per sphere (batch_grouped = 0): the same mean first passage times
    and capacitances, both to the requested residual, and fewer kernel launches grouped."""
    g = L.rng(79)
    inst = []
    for b in range(10):
        N = int(g.integers(20, 120))
        eps = float(g.uniform(0.02, 0.04))
        inst.append((L.uniform(N, eps, L.rng(79, b + 1)), eps, b % 2))
    kw = dict(npan=6, nord=10, ntheta_fine=24)
    out, launches = {}, {}
    for grouped in (1, 0):
        n0 = ncs.launch_count()
        out[grouped] = ncs.batch_solve(inst, 21, tol=1e-10, precision=ncs.MIXED, workers=4, batch_grouped=grouped, **kw)
        launches[grouped] = ncs.launch_count() - n0
        assert out[grouped]["rc"] == 0 and (out[grouped]["status"] == 0).all()
        assert (out[grouped]["relres"] <= 1e-10).all()
    d = np.abs(out[1]["scalar"] - out[0]["scalar"]) / np.abs(out[0]["scalar"])
    print(f"grouped vs separate: max relative difference {d.max():.2e}; launches {launches[1]} vs {launches[0]}")
    assert d.max() <= 1e-9
    assert launches[1] < launches[0]
