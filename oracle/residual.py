"""The L2 residual of the multiple-scattering system on one patch (Kaye & Greengard,
Section 9, eq. l2res): the discrepancy of the computed boundary values with the
Dirichlet data 1 on a patch Gamma_i,

    r(x) = S sigma_i(x) + sum_{j != i} S_ij sigma_j(x) - 1,   x on Gamma_i.

Test infrastructure only (see the package docstring).

  * S sigma_i = sum_k fhat_ik q_k: every basis density b_k solves the one-patch equation
    S b_k = q_k on its patch (Section 8), to the one-patch residual that the eq. patcherrl2
    check pins separately.
  * S_ij sigma_j for j != i by the fine-grid quadrature of patch j (Section 5): the points
    of Gamma_i are at least 2 eps from every other centre.
  * Reading of the printed normalisation: eq. l2res divides the L2 norm by |Gamma_i|; the
    text calls the quantity the relative L2 residual, which for data 1 is
    ||r|| / ||1|| = ||r|| / sqrt(|Gamma_i|), the root mean square of r over the patch. That
    is what is returned.
  * Quadrature on the patch: Gauss-Legendre in the arclength t on [0, eps] (measure
    sin t dt) times the trapezoidal rule in theta.
"""
import numpy as np

from . import zernike
from .geometry import local_to_global, patch_points
from .kernels import G_on_surface
from .quad import gauss_legendre


def patch_grid(pre, nt=None, nth=None):
    """(t, theta, dA) of the residual's quadrature on a patch: nt Gauss-Legendre nodes in t,
    nth angles; defaults resolve a degree-(M + 8) function."""
    M = pre.op.M
    nt = nt or M + 8
    nth = nth or 2 * M + 10
    t, wt = gauss_legendre(0.0, pre.eps, nt)
    th = 2.0 * np.pi * np.arange(nth) / nth
    T, TH = np.meshgrid(t, th, indexing="ij")
    dA = (wt * np.sin(t))[:, None] * np.full(nth, 2.0 * np.pi / nth)[None, :]
    return T.ravel(), TH.ravel(), dA.ravel()


def incoming_on_patch(pre, centres, fhat, i, t, th, chunk=4096):
    """u_i(x) = sum_{j != i} S_ij sigma_j at the points (t, theta) of patch i, by the
    fine-grid quadrature of every other patch."""
    centres = np.asarray(centres, dtype=np.float64)
    N, K = centres.shape[0], pre.K
    F = np.asarray(fhat, dtype=np.float64).reshape(N, K)
    x = local_to_global(centres[i], t, th)
    others = [j for j in range(N) if j != i]
    if not others:
        return np.zeros(x.shape[0])
    src = patch_points(centres[others], pre.op.t_f, pre.op.th_f).reshape(-1, 3)
    strength = (pre.op.w[None, :] * (F[others] @ pre.op.B.T)).reshape(-1)
    out = np.zeros(x.shape[0])
    for s in range(0, src.shape[0], chunk):
        diff = x[:, None, :] - src[None, s:s + chunk, :]
        d = np.sqrt(np.sum(diff * diff, axis=-1))
        out += G_on_surface(d, pre.mode) @ strength[s:s + chunk]
    return out


def residual_values(pre, centres, fhat, i, t, th):
    """r(x) at the points (t, theta) of patch i."""
    N = np.asarray(centres).shape[0]
    F = np.asarray(fhat, dtype=np.float64).reshape(N, pre.K)
    self_part = zernike.q_eval(pre.K, t / pre.eps, th) @ F[i]
    return self_part + incoming_on_patch(pre, centres, fhat, i, t, th) - 1.0


def patch_residual(pre, centres, fhat, i, nt=None, nth=None):
    """Relative L2 residual (root mean square of r over Gamma_i)."""
    t, th, dA = patch_grid(pre, nt, nth)
    r = residual_values(pre, centres, fhat, i, t, th)
    return float(np.sqrt(np.sum(dA * r * r) / np.sum(dA)))
