"""The discrete multiple-scattering operator (Kaye & Greengard, Sections 6-7).

Test infrastructure only (see the package docstring).

  * dense_operator: A = I + [P S_ij B]_{i != j} with S_ij(k, l) = G(x^z_{i,k}, x^f_{j,l}) w^f_l
    (eq. opinteqnsdisc); right-hand side b_i = P 1 (length K* vector of ones).
  * fine_matvec: the same product without forming A.
  * id_matvec: the compressed product of Section 7.1 without a tree:
    rho_j = T f_j (eq. Tmap), z_i(k) = sum_{j != i} sum_m G(x^z_{i,k}, x^f_{j,pi(m)}) rho_{j,m},
    y_i = f_i + P z_i.
"""
from dataclasses import dataclass

import numpy as np

from . import zernike
from .geometry import patch_points
from .idcomp import interpolative_decomposition
from .kernels import G_on_surface
from .onepatch import solve_one_patch


@dataclass
class Precompute:
    eps: float
    mode: int
    K: int
    op: object            # onepatch.OnePatch
    idr: object           # idcomp.IDResult or None
    P: np.ndarray         # K x K*
    r_z: np.ndarray       # Zernike nodes on the unit disk
    th_z: np.ndarray

    @property
    def Kstar(self):
        return self.r_z.size


def make_precompute(eps, mode, K, npan=13, nord=20, ntheta=None, tau=1e-11, with_id=True):
    """Step 1 of Section 7: one-patch solve, ID, T, I, P."""
    op = solve_one_patch(eps, mode, K, npan, nord, ntheta)
    idr = interpolative_decomposition(op, tau) if with_id else None
    P, r_z, th_z = zernike.transform(K)
    return Precompute(eps, mode, K, op, idr, P, r_z, th_z)


def zernike_points(pre, centres):
    return patch_points(centres, pre.eps * pre.r_z, pre.th_z)


def fine_points_all(pre, centres):
    return patch_points(centres, pre.op.t_f, pre.op.th_f)


def skeleton_points_all(pre, centres):
    return patch_points(centres, pre.idr.t_skel, pre.idr.th_skel)


def _pair_field(targets, sources, strengths, mode, chunk=2048):
    """sum over sources of G(target, source) * strength, for (n,3) targets."""
    out = np.zeros(targets.shape[0])
    for s in range(0, sources.shape[0], chunk):
        src = sources[s:s + chunk]
        diff = targets[:, None, :] - src[None, :, :]
        d = np.sqrt(np.sum(diff * diff, axis=-1))
        out += G_on_surface(d, mode) @ strengths[s:s + chunk]
    return out


def rhs(pre, N):
    """b_i = P 1 for every patch (eq. opinteqnsdisc)."""
    return np.tile(pre.P @ np.ones(pre.Kstar), N)


def dense_operator(pre, centres):
    """The KN x KN matrix I + [P S_ij B] (eq. opinteqnsdisc)."""
    N = len(centres)
    K = pre.K
    Z = zernike_points(pre, centres)
    F = fine_points_all(pre, centres)
    WB = pre.op.w[:, None] * pre.op.B
    A = np.eye(N * K)
    for i in range(N):
        for j in range(N):
            if i == j:
                continue
            diff = Z[i][:, None, :] - F[j][None, :, :]
            S = G_on_surface(np.sqrt(np.sum(diff * diff, axis=-1)), pre.mode)
            A[i * K:(i + 1) * K, j * K:(j + 1) * K] = pre.P @ (S @ WB)
    return A


def fine_matvec(pre, centres, x):
    """y = x + [P sum_{j != i} S_ij B x_j]_i without forming the matrix."""
    N = len(centres)
    K = pre.K
    X = np.asarray(x, dtype=np.float64).reshape(N, K)
    Z = zernike_points(pre, centres)
    F = fine_points_all(pre, centres)
    dens = (pre.op.B @ X.T).T * pre.op.w[None, :]     # N x n_f: sigma_j * w
    Y = X.copy()
    for i in range(N):
        z = np.zeros(pre.Kstar)
        for j in range(N):
            if j != i:
                z += _pair_field(Z[i], F[j], dens[j], pre.mode)
        Y[i] += pre.P @ z
    return Y.ravel()


def outgoing(pre, x, N):
    """rho_j = T f_j for every patch, (N, p) (eq. Tmap)."""
    X = np.asarray(x, dtype=np.float64).reshape(N, pre.K)
    return X @ pre.idr.T.T


def id_field(pre, centres, x, patches=None):
    """z_i at the Zernike nodes of the selected patches via the compressed sums
    (no tree). Returns (len(patches), K*)."""
    N = len(centres)
    rho = outgoing(pre, x, N)
    S = skeleton_points_all(pre, centres)
    Z = zernike_points(pre, centres)
    patches = range(N) if patches is None else patches
    out = []
    for i in patches:
        if N == 1:
            out.append(np.zeros(pre.Kstar))
            continue
        src = np.concatenate([S[j] for j in range(N) if j != i])
        st = np.concatenate([rho[j] for j in range(N) if j != i])
        out.append(_pair_field(Z[i], src, st, pre.mode))
    return np.array(out)


def id_matvec(pre, centres, x):
    """y = x + P z with z from the compressed sums (Section 7.1, no tree)."""
    N = len(centres)
    z = id_field(pre, centres, x)
    return (np.asarray(x, float).reshape(N, pre.K) + z @ pre.P.T).ravel()
