"""Host-side logic of the C-ABI library, checked on CPU against the oracle: symbol
exports, one-patch precompute (B, I, P), the library's own ID/outgoing operator, and
input validation. No GPU call is made here."""
import re
import os

import numpy as np
import pytest

from oracle import onepatch, zernike, idcomp
from oracle.kernels import G_on_surface, chord, EXTERIOR, INTERIOR
from paper_1906_04209_gb300 import ncs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_exports_match_header(libncs):
    hdr = open(os.path.join(ROOT, "include", "ncs.h")).read()
    names = set(re.findall(r"\b(ncs_[a-z0-9_]+)\s*\(", hdr))
    assert names, "no declarations found"
    for n in names:
        assert hasattr(libncs, n), n
    assert set(ncs.EXPORTS) == names


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_onepatch_matches_oracle(libncs, mode):
    eps, K, npan, nord, nth = 0.05, 21, 7, 12, 30
    c = ncs.Context(eps, mode, K, npan=npan, nord=nord, ntheta_fine=nth)
    tr, beta = c.onepatch()
    op = onepatch.solve_one_patch(eps, mode, K, npan, nord, nth)
    assert np.abs(tr - op.rad.t).max() < 1e-15
    assert np.abs(beta - op.beta).max() < 1e-11 * np.abs(op.beta).max()
    o = c.operator()
    assert np.abs(o["I"] - op.I).max() < 1e-11 * np.abs(op.I).max()
    P, r, th = zernike.transform(K)
    assert np.abs(o["P"] - P).max() < 1e-13
    assert np.abs(o["znode_r"] - r).max() < 1e-15 and np.abs(o["znode_theta"] - th).max() < 1e-15


def test_precompute_independent_of_thread_count(libncs):
    """The host precompute splits its loops over threads by rows, columns and modes, never
    inside a sum: one thread and all threads give the same bits."""
    kw = dict(npan=6, nord=10, ntheta_fine=24, device_precompute=0, id_ladder_max=0.2)
    a = ncs.Context(0.05, INTERIOR, 21, threads=1, **kw)
    b = ncs.Context(0.05, INTERIOR, 21, threads=0, **kw)
    assert np.array_equal(a.onepatch()[1], b.onepatch()[1])
    oa, ob = a.operator(), b.operator()
    assert np.array_equal(oa["T"], ob["T"]) and np.array_equal(oa["I"], ob["I"])
    assert np.array_equal(a.reps()[1], b.reps()[1])


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_library_outgoing_operator(libncs, mode):
    """The library's own ID (sketched CPQR) reproduces the far field of the oracle's
    fine-grid quadrature (eq. outgoingcompressed) at held-out far targets."""
    eps, K = 0.05, 21
    c = ncs.Context(eps, mode, K, npan=7, nord=12, ntheta_fine=30)
    o = c.operator()
    op = onepatch.solve_one_patch(eps, mode, K, 7, 12, 30)
    xt = idcomp.training_grid(eps, 1e-11, nper=5, rho_min_factor=2.07)
    xf = idcomp.fine_points(op)
    st, sth = o["skel_t"], o["skel_theta"]
    xs = np.stack([np.sin(st) * np.cos(sth), np.sin(st) * np.sin(sth), np.cos(st)], 1)
    f = np.random.default_rng(5).standard_normal(K)
    ref = G_on_surface(chord(xt[:, None], xf[None]), mode) @ (op.w * (op.B @ f))
    lib = G_on_surface(chord(xt[:, None], xs[None]), mode) @ (o["T"] @ f)
    assert np.abs(lib - ref).max() < 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_library_id_ladder_accuracy(libncs, mode):
    """Every representation of the library's ID ladder (far fields beyond
    2, 2.52, 3.17, 4, ... eps) reproduces the fine-grid far field at held-out targets beyond its radius."""
    eps, K = 0.02, 21
    c = ncs.Context(eps, mode, K, npan=7, nord=12, ntheta_fine=30, id_ladder_max=0.5)
    op = onepatch.solve_one_patch(eps, mode, K, 7, 12, 30)
    xf = idcomp.fine_points(op)
    f = np.random.default_rng(6).standard_normal(K)
    src = op.w * (op.B @ f)
    rm, ps = c.reps()
    assert len(ps) >= 6
    for r in range(len(ps)):
        T, st, sth = c.rep(r)
        xt = idcomp.training_grid(eps, 1e-11, nper=5, rho_min_factor=1.03 * rm[r] / eps)
        xs = np.stack([np.sin(st) * np.cos(sth), np.sin(st) * np.sin(sth), np.cos(st)], 1)
        ref = G_on_surface(chord(xt[:, None], xf[None]), mode) @ src
        lib = G_on_surface(chord(xt[:, None], xs[None]), mode) @ (T @ f)
        assert np.abs(lib - ref).max() < 1e-9 * np.abs(ref).max(), (r, rm[r], ps[r])


def test_set_precision_validation(libncs):
    c = ncs.Context(0.05, INTERIOR, 10, npan=6, nord=10, ntheta_fine=24)
    for p in (ncs.FP64, ncs.FP32, ncs.MIXED, ncs.DF64):
        c.set_precision(p)
    for bad in (-1, 4, 99):
        with pytest.raises(ncs.NcsError):
            c.set_precision(bad)


def test_create_validation(libncs):
    for args in [(0.0, 0, 10), (1.5, 0, 10), (0.1, 2, 10), (0.1, 0, 0)]:
        with pytest.raises(ncs.NcsError) as e:
            ncs.Context(*args, npan=4, nord=6)
        assert e.value.code == ncs.NCS_E_INPUT


def test_inner_grid_tol_validation(libncs):
    """inner_grid_tol (the mixed solve's inner tree) accepts 0 (off) up to below 0.1; the
    context reports no inner tree before one is built."""
    assert ncs.default_params().inner_grid_tol == 1e-5
    for bad in (-1e-6, 0.1, 0.5):
        with pytest.raises(ncs.NcsError) as e:
            ncs.Context(0.1, 1, 3, npan=4, nord=6, inner_grid_tol=bad)
        assert e.value.code == ncs.NCS_E_INPUT
    for ok in (0.0, 1e-9, 1e-3):
        c = ncs.Context(0.1, 1, 3, npan=4, nord=6, ntheta_fine=8, inner_grid_tol=ok)
        info = c.info()
        assert info["inner_grid_points"] == 0 and info["inner_tree_pairs"] == 0


def test_set_patches_validation(libncs):
    c = ncs.Context(0.1, 1, 3, npan=4, nord=6, ntheta_fine=8)
    with pytest.raises(ncs.NcsError) as e:  # geodesic distance 0.25 < 3 eps
        c.set_patches([[0, 0, 1.0], [np.sin(0.25), 0, np.cos(0.25)]])
    assert e.value.code == ncs.NCS_E_INPUT
    with pytest.raises(ncs.NcsError) as e:
        c.set_patches([[0, 0, 1.1]])
    assert e.value.code == ncs.NCS_E_INPUT
    c.set_patches([[0, 0, 1.0], [np.sin(0.31), 0, np.cos(0.31)]])
    assert c.info()["N"] == 2
    with pytest.raises(ncs.NcsError) as e:  # arguments are checked before any device work
        c.solve(tol=0)
    assert e.value.code == ncs.NCS_E_INPUT


def test_separation_check_names_the_first_pair(libncs):
    # the check runs over all patches in parallel and reports the first offending patch in
    # index order with its partner, as a serial scan would
    from paper_1906_04209_gb300 import layouts as L
    eps = 0.005
    c = L.uniform(5000, eps, L.rng(77))
    a, b = 1234, 3000
    # move patch b to 2 eps (geodesic) from patch a, along a tangent direction of a
    t = np.cross(c[a], [0.0, 0.0, 1.0])
    t /= np.linalg.norm(t)
    c[b] = np.cos(2 * eps) * c[a] + np.sin(2 * eps) * t
    # keep the layout otherwise valid: drop patches that the move brought too close to b
    d = np.arccos(np.clip(c @ c[b], -1, 1))
    keep = [i for i in range(len(c)) if i in (a, b) or d[i] >= 3 * eps]
    c = c[keep]
    ia, ib = keep.index(a), keep.index(b)
    ctx = ncs.Context(eps, 1, 3, npan=4, nord=6, ntheta_fine=8)
    with pytest.raises(ncs.NcsError) as e:
        ctx.set_patches(c)
    assert e.value.code == ncs.NCS_E_INPUT
    assert f"patches {min(ia, ib)} and {max(ia, ib)} are closer than 3 eps" in str(e.value)


def test_precompute_without_device_uses_host_sketch(libncs):
    # without a CUDA device the ID sketch and the collocation matrices are formed on the host
    # whatever the parameter says
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    c = ncs.Context(0.05, INTERIOR, 10, npan=6, nord=10, ntheta_fine=24, device_precompute=1)
    t = c.timings()
    assert t[2] == 0.0 and t[6] == 0.0
    assert t[7] > 0.0 and t[8] >= 0.0 and t[7] + t[8] <= t[0] + 1e-9


def test_launch_count_without_gpu(libncs):
    # no kernel has been launched by the CPU-only tests; the counter is readable anyway
    assert ncs.launch_count() >= 0


def test_id_ladder_max(libncs):
    """id_ladder_max = 0 keeps only the far-field-beyond-2-eps representation; a larger
    radius adds the ladder (more, smaller representations, decreasing p)."""
    kw = dict(npan=6, nord=10, ntheta_fine=24)
    one = ncs.Context(0.05, INTERIOR, 10, id_ladder_max=0.0, **kw)
    rm1, p1 = one.reps()
    assert len(p1) == 1 and abs(rm1[0] - 2 * 0.05) < 1e-12
    lad = ncs.Context(0.05, INTERIOR, 10, id_ladder_max=0.5, **kw)
    rm, ps = lad.reps()
    # the training grids differ (panel edges at the ladder radii), so the rank of the
    # 2 eps representation may move by a few points
    assert len(ps) > 1 and abs(int(ps[0]) - int(p1[0])) <= 4
    assert all(ps[i] >= ps[i + 1] for i in range(len(ps) - 1))
    assert rm.max() <= 0.5 + 1e-12
    with pytest.raises(ncs.NcsError):
        ncs.Context(0.05, INTERIOR, 10, id_ladder_max=-1.0, **kw)


def test_tuning_validation(libncs):
    """ncs_set_tuning accepts the documented ranges only; ncs_tune needs patches first."""
    c = ncs.Context(0.05, INTERIOR, 10, npan=6, nord=10, ntheta_fine=24)
    t0 = c.get_tuning()
    assert t0 == dict(p2l_tile=16, p2l_poly=4, direct_poly=4, item_patches=16, l2p_weight=0.1, p2l_rsq=0,
                      direct_rsq=0)
    c.set_tuning(p2l_tile=8, p2l_poly=2, direct_poly=6, item_patches=32, l2p_weight=0.2, p2l_rsq=4, direct_rsq=8)
    assert c.get_tuning() == dict(p2l_tile=8, p2l_poly=2, direct_poly=6, item_patches=32, l2p_weight=0.2,
                                  p2l_rsq=4, direct_rsq=8)
    for bad in (dict(p2l_tile=12), dict(p2l_poly=3), dict(direct_poly=8), dict(item_patches=4),
                dict(p2l_tile=16, item_patches=24), dict(l2p_weight=0.0), dict(p2l_rsq=2), dict(direct_rsq=6)):
        with pytest.raises(ncs.NcsError) as e:
            c.set_tuning(**bad)
        assert e.value.code == ncs.NCS_E_INPUT
    with pytest.raises(ncs.NcsError) as e:
        c.tune(flags=3)
    assert e.value.code == ncs.NCS_E_STATE
