"""Pins of the oracle's multiple-scattering operator, solve and outputs
(eq. opinteqnsdisc, Section 7.1, GMRES, eqs. getI and mufromsigma2)."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import idcomp, solve as S, operator as O
from oracle.kernels import EXTERIOR, INTERIOR, G_on_surface
from paper_1906_04209_gb300 import layouts as L


def _centres(N, eps, seed):
    return L.uniform(N, eps, L.rng(90, seed))


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_dense_equals_matrix_free(small_pre, mode):
    pre = small_pre(mode)
    c = _centres(5, 0.1, 1)
    x = np.random.default_rng(0).standard_normal(5 * pre.K)
    A = O.dense_operator(pre, c)
    assert np.abs(A @ x - O.fine_matvec(pre, c, x)).max() < 1e-12 * np.abs(A @ x).max()


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_compressed_equals_dense(small_pre, mode):
    """The ID-compressed product agrees with eq. opinteqnsdisc to the ID tolerance."""
    pre = small_pre(mode)
    c = _centres(6, 0.1, 2)
    x = np.random.default_rng(1).standard_normal(6 * pre.K)
    y = O.dense_operator(pre, c) @ x
    assert np.abs(O.id_matvec(pre, c, x) - y).max() < 1e-9 * np.abs(y).max()


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_id_error_held_out(small_pre, mode):
    """||A - A~ Pi|| on a held-out far-field grid is O(tau) (Section 7.1, eq. idapprox)."""
    pre = small_pre(mode)
    xt = idcomp.training_grid(pre.eps, 1e-11, nper=7, rho_min_factor=2.03)
    assert idcomp.id_error(pre.op, pre.idr, xt) < 1e-9


def test_single_patch_is_identity(small_pre):
    """N = 1: no scattering, f = P 1 exactly."""
    pre = small_pre(INTERIOR)
    c = np.array([[0.0, 0.6, 0.8]])
    b = O.rhs(pre, 1)
    assert np.abs(O.id_matvec(pre, c, b) - b).max() < 1e-15


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_gmres_matches_lu(small_pre, mode):
    pre = small_pre(mode)
    N = 6
    c = _centres(N, 0.1, 3)
    A = O.dense_operator(pre, c)
    b = O.rhs(pre, N)
    x_lu = S.dense_solve(A, b)
    x, it, hist, true = S.gmres(lambda v: A @ v, b, 1e-13)
    assert np.abs(x - x_lu).max() < 1e-12 * np.abs(x_lu).max()
    assert true < 1e-12
    assert np.all(np.diff(hist) <= 1e-15)  # GMRES residual is monotone
    assert it <= N * pre.K


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_rotation_and_permutation_invariance(small_pre, mode):
    """mu / C under rigid motions and relabelling. A rotation about the z axis carries
    every patch frame with it (e1 = z x c / |z x c|), so the discrete system is
    unchanged up to rounding; a general rotation turns each frame about its centre,
    which moves the Zernike sampling nodes, so the result changes only at the level
    of the Zernike truncation error; relabelling is exact."""
    pre = small_pre(mode, ntheta=44)
    N = 5
    c = _centres(N, 0.1, 4)
    out = []
    Rz = Rotation.from_rotvec([0.0, 0.0, 1.234]).as_matrix()
    R = Rotation.from_rotvec([0.3, -1.1, 0.7]).as_matrix()
    perm = np.array([3, 0, 4, 1, 2])
    for cc in (c, c @ Rz.T, c[perm], c @ R.T):
        A = O.dense_operator(pre, cc)
        x = S.dense_solve(A, O.rhs(pre, N))
        out.append(S.outputs(pre.op.I, x, N, mode)[1])
    assert abs(out[1] - out[0]) < 1e-12 * abs(out[0])
    assert abs(out[2] - out[0]) < 1e-12 * abs(out[0])
    assert abs(out[3] - out[0]) < 1e-7 * abs(out[0])


def test_output_formula_limits():
    """Full coverage with a uniform density: int G_I sigma = 1 gives sigma = 1/(8 pi),
    I = 1/2 and mu = 1/15 (the fully absorbing ball, mean of (1 - r^2)/6); the exterior
    gives I = 1 and C = 4 pi (unit-sphere capacitance)."""
    from scipy.integrate import quad
    for mode, expect in ((INTERIOR, 1 / 15), (EXTERIOR, 4 * np.pi)):
        mean = quad(lambda r: G_on_surface(2 * np.sin(r / 2), mode) * np.sin(r), 0, np.pi, limit=200)[0] / 2
        sigma = 1.0 / (4 * np.pi * mean)
        Is = 4 * np.pi * sigma
        _, val = S.outputs(np.array([Is]), np.array([1.0]), 1, mode)
        assert abs(val - expect) < 1e-12 * expect


@pytest.mark.parametrize("mode", [EXTERIOR, INTERIOR])
def test_point_charge_limit(mode):
    """Well-separated small patches: the solve matches the point-charge model
    q_i / Q1 + sum_{j != i} G(c_i, c_j) q_j = 1 with the one-patch charge Q1 (the
    same small-eps expansion as the one-patch test) to relative O(eps^2)."""
    eps, N, K = 0.005, 4, 3
    pre = O.make_precompute(eps, mode, K, npan=8, nord=10, ntheta=12, tau=1e-12)
    c = np.array([[0, 0, 1.0], [1.0, 0, 0], [0, 1.0, 0], [-0.6, -0.64, 0.48]])
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    A = O.dense_operator(pre, c)
    x = S.dense_solve(A, O.rhs(pre, N))
    Is, _ = S.outputs(pre.op.I, x, N, mode)
    Q1 = pre.op.I[0] * np.sqrt(np.pi)
    M = np.eye(N) / Q1
    for i in range(N):
        for j in range(N):
            if i != j:
                M[i, j] = G_on_surface(np.linalg.norm(c[i] - c[j]), mode)
    q = np.linalg.solve(M, np.ones(N))
    assert abs(q.sum() - Is) < 20 * eps ** 2 * Is
