"""The GMRES solve (Section 7, Step 3) with its state on the device: the captured
CUDA-graph step against the same kernels launched one by one, against the oracle's
solve, and the error paths of ncs_solve and ncs_batch_solve (iteration cap, FP32
estimate below a tolerance its product cannot reach, overflow in the operator, one
corrupted instance in a batch). Failures are made on the host (inputs, caps), never by
faulting the device."""
import numpy as np
import pytest

from oracle import operator as O, solve as S
from oracle.kernels import EXTERIOR, INTERIOR
from paper_1906_04209_gb300 import layouts as L, ncs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda(libncs):
    assert torch.cuda.is_available(), "GPU test without a GPU"
    torch.cuda.set_device(0)


def _ctx(pre, T_max=None, **kw):
    T = pre.idr.T if T_max is None else (pre.idr.T / np.abs(pre.idr.T).max()) * T_max
    return ncs.Context(pre.eps, pre.mode, pre.K,
                       operator=(T, pre.idr.t_skel, pre.idr.th_skel, pre.op.I), **kw)


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_graph_step_equals_direct_launches(small_pre, mode):
    """Replaying the captured step runs the same kernels in the same order: iterates are
    bitwise equal, and both match the oracle's GMRES on the compressed operator."""
    pre = small_pre(mode)
    N = 30
    c = L.uniform(N, pre.eps, L.rng(93, mode))
    out = {}
    for graphs in (0, 1):
        ctx = _ctx(pre, method=ncs.METHOD_DIRECT, cuda_graphs=graphs)
        ctx.set_patches(c)
        r = ctx.solve(tol=1e-12, precision=ncs.FP64)
        st = ctx.solve_stats()
        assert (st["graph_replays"] > 0) == bool(graphs)
        assert st["recomputed"] == 1.0 and st["relres"] == r["relres"]
        assert st["gmres_steps"] + st["residual_products"] == r["iterations"]
        out[graphs] = r
    assert np.array_equal(out[0]["fhat"], out[1]["fhat"])
    assert out[0]["iterations"] == out[1]["iterations"]
    b = O.rhs(pre, N)
    xr, _, _, _ = S.gmres(lambda v: O.id_matvec(pre, c, v), b, 1e-13)
    assert np.abs(out[1]["fhat"] - xr).max() <= 1e-10 * np.abs(xr).max()


def test_graph_step_tree_mixed(small_pre):
    """The mixed solve on the tree replays its FP32 step graph across refinement steps
    and gives the same answer as direct launches (to rounding: the P2L kernel adds its
    partial sums into the grids atomically, so two runs differ in the last bits); its
    reported residual is recomputed."""
    eps = 0.01
    pre = small_pre(INTERIOR, eps=eps)
    N = 2500
    c = L.uniform(N, eps, L.rng(94))
    res = {}
    for graphs in (0, 1):
        ctx = _ctx(pre, method=ncs.METHOD_TREE, cuda_graphs=graphs)
        ctx.set_patches(c)
        r = ctx.solve(tol=1e-9, precision=ncs.MIXED)
        st = ctx.solve_stats()
        assert r["relres"] <= 1e-9 and st["recomputed"] == 1.0
        assert st["refinement_steps"] >= 1
        res[graphs] = (r, st)
    f0, f1 = res[0][0]["fhat"], res[1][0]["fhat"]
    assert np.abs(f0 - f1).max() <= 1e-9 * np.abs(f0).max()
    assert res[1][1]["graph_replays"] > 0 and res[0][1]["graph_replays"] == 0


def test_iteration_cap_returns_noconv(small_pre):
    pre = small_pre(INTERIOR)
    N = 20
    c = L.uniform(N, pre.eps, L.rng(95))
    ctx = _ctx(pre, method=ncs.METHOD_DIRECT, gmres_maxit=2)
    ctx.set_patches(c)
    r = ctx.solve(tol=1e-14, precision=ncs.FP64, allow_noconv=True)
    assert r["rc"] == ncs.NCS_E_NOCONV
    # the outputs hold the last iterate: two GMRES steps and the recomputed residual
    assert r["iterations"] == 3
    assert np.all(np.isfinite(r["fhat"])) and np.abs(r["fhat"]).max() > 0
    assert 1e-14 < r["relres"] < 1.0
    with pytest.raises(ncs.NcsError) as e:
        ctx.solve(tol=1e-14, precision=ncs.FP64)
    assert e.value.code == ncs.NCS_E_NOCONV


def test_fp32_solve_does_not_claim_unreachable_tolerance(small_pre):
    """An FP32-product solve at 1e-11: its GMRES estimate can fall below the tolerance
    while b - A x stays at the FP32 level; the solve must then report NOCONV."""
    pre = small_pre(EXTERIOR)
    N = 40
    c = L.uniform(N, pre.eps, L.rng(96, 1))
    ctx = _ctx(pre, method=ncs.METHOD_DIRECT)
    ctx.set_patches(c)
    r = ctx.solve(tol=1e-11, precision=ncs.FP32, allow_noconv=True)
    assert (r["rc"] == ncs.NCS_E_NOCONV) or (r["relres"] <= 1e-11)
    assert r["rc"] == ncs.NCS_E_NOCONV  # FP32 products cannot give a 1e-11 residual


def test_overflowing_operator_returns_numeric(small_pre):
    """An outgoing operator with entries near the FP64 overflow threshold (finite, so it
    passes input validation) makes the Arnoldi vector non-finite: NCS_E_NUMERIC."""
    pre = small_pre(INTERIOR)
    N = 12
    c = L.uniform(N, pre.eps, L.rng(97, 1))
    assert np.all(np.isfinite((pre.idr.T / np.abs(pre.idr.T).max()) * 1e307))
    ctx = _ctx(pre, T_max=1e307, method=ncs.METHOD_DIRECT)
    ctx.set_patches(c)
    with pytest.raises(ncs.NcsError) as e:
        ctx.solve(tol=1e-10, precision=ncs.FP64)
    assert e.value.code == ncs.NCS_E_NUMERIC
    # the context stays usable: a correct operator on a new context still solves
    ok = _ctx(pre, method=ncs.METHOD_DIRECT)
    ok.set_patches(c)
    assert ok.solve(tol=1e-10, precision=ncs.FP64)["relres"] <= 1e-10


def test_batch_with_one_corrupted_instance():
    """One instance's centres hold a NaN (a host-side corruption): that instance fails
    input validation and every other instance still converges."""
    g = L.rng(79)
    inst = []
    for b in range(5):
        N = int(g.integers(20, 120))
        eps = float(g.uniform(0.02, 0.04))
        inst.append((L.uniform(N, eps, L.rng(79, b + 1)), eps, b % 2))
    bad = inst[2][0].copy()
    bad[3, 1] = np.nan
    inst[2] = (bad, inst[2][1], inst[2][2])
    kw = dict(npan=6, nord=10, ntheta_fine=24, method=ncs.METHOD_DIRECT)
    out = ncs.batch_solve(inst, 21, tol=1e-10, precision=ncs.MIXED, workers=2, **kw)
    assert out["status"][2] == ncs.NCS_E_INPUT
    assert out["rc"] == ncs.NCS_E_INPUT
    for b in (0, 1, 3, 4):
        assert out["status"][b] == 0 and out["relres"][b] <= 1e-10
