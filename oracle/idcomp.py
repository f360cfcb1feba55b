"""Interpolative decomposition of the outgoing field (Kaye & Greengard, Section 7.1).

Test infrastructure only (see the package docstring).

Steps:
  1. A training grid x^t on the far-field region Theta = {points farther than
     2 eps (arclength) from the patch centre}; the paper leaves the grid open.
     Reading: geodesic polar grid about the centre, radial panels
     [2e, 4e], [4e, 8e], ... up to pi with Gauss-Legendre nodes, and on each panel
     [a, b] an azimuthal count 2 m + 1 with (eps/a)^m below tau/10, because a
     field generated inside the patch decays like (eps/rho)^m in azimuthal mode m.
  2. A[j, l] = G(x^t_j, x^f_l).
  3. Column-pivoted QR (LAPACK via scipy) A P = Q R; rank p = first k with
     |R_kk| < tau |R_00|; Pi = [I, R11^-1 R12] in pivoted order; pi(m) = first p
     pivots.
  4. T = Pi W B (eq. Tmap).
"""
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from .kernels import G_on_surface, chord
from .quad import gauss_legendre


def training_grid(eps, tau, nper=10, rho_min_factor=2.0):
    """Training points on the far-field region, patch centred at the north pole.
    Returns an (n_t, 3) array."""
    edges = [rho_min_factor * eps]
    while edges[-1] * 2.0 < np.pi:
        edges.append(edges[-1] * 2.0)
    edges.append(np.pi)
    pts = []
    for a, b in zip(edges[:-1], edges[1:]):
        rho, _ = gauss_legendre(a, b, nper)
        m = int(np.ceil(np.log(tau / 10.0) / np.log(eps / a)))
        m = max(m, 8)
        nphi = 2 * m + 1
        phi = 2.0 * np.pi * np.arange(nphi) / nphi
        R, P = np.meshgrid(rho, phi, indexing="ij")
        R = R.ravel()
        P = P.ravel()
        pts.append(np.stack([np.sin(R) * np.cos(P), np.sin(R) * np.sin(P), np.cos(R)], 1))
    return np.concatenate(pts)


def fine_points(op):
    """Fine-grid points of the generic patch at the north pole, (n_f, 3)."""
    t, th = op.t_f, op.th_f
    return np.stack([np.sin(t) * np.cos(th), np.sin(t) * np.sin(th), np.cos(t)], 1)


@dataclass
class IDResult:
    p: int
    skel: np.ndarray      # indices pi(m) into the fine grid, length p
    Pi: np.ndarray        # p x n_f
    T: np.ndarray         # p x K
    t_skel: np.ndarray    # local (t, theta) of the skeleton points
    th_skel: np.ndarray
    rdiag: np.ndarray


def interpolative_decomposition(op, tau, nper=10, rho_min_factor=2.0):
    """ID of the training matrix and the outgoing map T = Pi W B, for the far field
    beyond rho_min_factor * eps (2 eps in Section 7.1; larger values give the coarser
    per-level representations of "Optimizations and parallelization")."""
    xt = training_grid(op.eps, tau, nper, rho_min_factor)
    xf = fine_points(op)
    A = G_on_surface(chord(xt[:, None, :], xf[None, :, :]), op.mode)
    R, piv = sla.qr(A, mode="r", pivoting=True, check_finite=False)
    if isinstance(R, tuple):
        R = R[0]
    d = np.abs(np.diag(R))
    small = np.nonzero(d < tau * d[0])[0]
    p = int(small[0]) if small.size else d.size
    R11 = R[:p, :p]
    R12 = R[:p, p:]
    X = sla.solve_triangular(R11, R12, check_finite=False)
    nf = A.shape[1]
    Pi = np.zeros((p, nf))
    Pi[:, piv[:p]] = np.eye(p)
    Pi[:, piv[p:]] = X
    T = Pi @ (op.w[:, None] * op.B)
    skel = piv[:p].copy()
    return IDResult(p, skel, Pi, T, op.t_f[skel], op.th_f[skel], d)


def id_error(op, idr, xt):
    """max |A - A~ Pi| / max |A| on the target points xt (held-out grid check)."""
    xf = fine_points(op)
    A = G_on_surface(chord(xt[:, None, :], xf[None, :, :]), op.mode)
    Ask = A[:, idr.skel]
    return float(np.abs(A - Ask @ idr.Pi).max() / np.abs(A).max())
