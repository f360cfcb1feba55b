"""Host logic of the cube-sphere quadtree (Section 7.2): the covering invariant of
the note in Step 3 (each ordered pair of distinct patches is accounted for exactly
once), on layouts that stress cube edges and corners, clusters and uniform spreads."""
import numpy as np
import pytest

from paper_1906_04209_gb300 import layouts as L, ncs


def _check(c, eps):
    ctx = ncs.Context(eps, 1, 3, npan=4, nord=6, ntheta_fine=8)
    ctx.set_patches(c)
    tg, sr, lv, kd = ctx.tree_pairs()
    N = len(c)
    key = tg.astype(np.int64) * N + sr
    u, cnt = np.unique(key, return_counts=True)
    assert (tg != sr).all()
    assert len(u) == N * (N - 1) and cnt.max() == 1
    # interaction-list pairs are never neighbours at their level: their boxes are
    # separated, so the centres are at least one box apart
    return lv.max() + 1


def _corner_layout(eps, seed):
    rng = np.random.default_rng(seed)
    keep = []
    for v in [(1, 1, 1), (1, 1, 0), (1, 0, 1), (-1, 1, 1), (1, -1, -1), (0, 1, 1), (-1, -1, -1), (0, 0, 1)]:
        v = np.array(v, float) / np.linalg.norm(v)
        for _ in range(25):
            p = v + 0.05 * rng.standard_normal(3)
            p /= np.linalg.norm(p)
            if all(np.arccos(np.clip(p @ q, -1, 1)) >= 3 * eps for q in keep):
                keep.append(p)
    return np.array(keep)


@pytest.mark.parametrize("name", ["uniform", "vmf", "corners", "fibonacci", "tiny"])
def test_covering_invariant(libncs, name):
    if name == "uniform":
        c, eps = L.uniform(600, 0.01, L.rng(11)), 0.01
    elif name == "vmf":
        c, eps = L.vmf_clusters(900, 0.002, L.rng(12)), 0.002
    elif name == "corners":
        eps = 0.003
        c = _corner_layout(eps, 13)
    elif name == "fibonacci":
        c, eps = L.jittered_fibonacci(1500, 0.003, L.rng(14)), 0.003
    else:
        c, eps = L.uniform(2, 0.1, L.rng(15)), 0.1
    assert _check(c, eps) >= 1


def test_tree_statistics(libncs):
    """Work counts follow the construction: the direct and grid parts together cover
    N (N - 1) patch pairs, and grids exist once groups hold several patches."""
    c, eps = L.uniform(3000, 0.005, L.rng(16)), 0.005
    ctx = ncs.Context(eps, 0, 10, npan=4, nord=6, ntheta_fine=12, method=ncs.METHOD_TREE)
    ctx.set_patches(c)
    s = ctx.tree_stats()
    info = ctx.info()
    assert s["grid_groups"] > 0 and s["grid_points"] > 0 and s["levels"] >= 4
    # every direct pair uses a representation no larger than the finest one
    assert 0 < s["direct_pairs"] <= s["direct_patch_pairs"] * info["p"] * info["Kstar"]
    assert s["p2l_pairs"] + s["direct_pairs"] < info["direct_pairs"]


def test_tree_build_independent_of_thread_count(libncs):
    """The tree's group plans are formed in parallel and merged in group order: one host
    thread and all of them build the same lists (same counts of grid groups, work items,
    pairs and transfers)."""
    c, eps, mode, _ = L.workload(2)
    stats = []
    for threads in (1, 0):
        ctx = ncs.Context(eps, mode, 3, npan=4, nord=6, ntheta_fine=8, threads=threads,
                          method=ncs.METHOD_TREE)
        ctx.set_patches(c)
        stats.append(ctx.tree_stats())
    assert stats[0] == stats[1]
    assert stats[0]["grid_groups"] > 0 and stats[0]["p2l_items"] > 0


def test_looser_grids_keep_the_covering(libncs):
    """The mixed solve's inner tree is the same construction at a looser incoming-grid
    tolerance: every ordered pair is still accounted for exactly once, with the same levels,
    fewer grid points and fewer P2L pair evaluations (groups may trade direct sums for grids,
    never drop a pair)."""
    c, eps = L.jittered_fibonacci(3000, 0.003, L.rng(17)), 0.003
    stats = {}
    for gt in (1e-8, 1e-5):
        ctx = ncs.Context(eps, 1, 3, npan=4, nord=6, ntheta_fine=8, grid_tol=gt, method=ncs.METHOD_TREE)
        ctx.set_patches(c)
        tg, sr, lv, kd = ctx.tree_pairs()
        N = len(c)
        u, cnt = np.unique(tg.astype(np.int64) * N + sr, return_counts=True)
        assert len(u) == N * (N - 1) and cnt.max() == 1
        stats[gt] = ctx.tree_stats()
    loose, fine = stats[1e-5], stats[1e-8]
    assert loose["levels"] == fine["levels"]
    assert loose["grid_points"] < fine["grid_points"]
    assert loose["p2l_pairs"] < fine["p2l_pairs"]
