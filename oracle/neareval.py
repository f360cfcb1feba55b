"""Single-layer potential of the patch densities at points off the sphere, including points
close to a patch (Kaye & Greengard, Section 2, eqs. urep and intBVPansatz with the
off-surface Green's functions eqs. Gextoffsurface / Gintoffsurface; the paper plots the
mean first passage time on the sphere of radius 1 - eps/5, Section 9.2).

Test infrastructure only (see the package docstring).

  * A patch farther than 2.5 eps (geodesic, from the target's radial projection) is summed
    with its fine-grid quadrature (Section 5), accurate there.
  * A nearer patch is integrated directly: sigma_j(t, theta) = sum_k fhat_jk beta_k(t)
    trig_k(theta) with beta_k interpolated on its radial panels (on the last panel through
    g = sigma sqrt(eps - t) and the substitution t = eps - u^2), the panels' rules graded
    toward the target's projection t0, and for every radial node a theta rule graded toward
    the target's azimuth theta0 on the scale of its distance to that circle.
"""
import numpy as np

from . import zernike
from .geometry import frame, local_to_global, patch_points
from .kernels import EXTERIOR, G_off_surface
from .onepatch import _panel_rule
from .quad import graded_toward


def _target_local(c, x):
    """(t0, theta0, r) of the target x in the polar frame of the patch centred at c."""
    e1, e2, e3 = frame(c)
    r = np.sqrt(x @ x)
    u = x / r
    t0 = np.arctan2(np.sqrt((u @ e1) ** 2 + (u @ e2) ** 2), u @ e3)
    th0 = np.arctan2(u @ e2, u @ e1)
    return t0, th0, r


def _theta_rule(th0, t, t0, delta):
    """Nodes and weights on [th0 - pi, th0 + pi] graded toward th0 on both sides, down to
    the angular scale of the target's distance to the circle t."""
    scale = np.sqrt(delta * delta + (t - t0) ** 2) / max(np.sin(t), 1e-300)
    nlev = int(min(50, max(1, np.ceil(np.log2(np.pi / max(scale, 1e-300))) + 3)))
    x1, w1 = graded_toward(th0 - np.pi, th0, th0, nlev, 12)
    x2, w2 = graded_toward(th0, th0 + np.pi, th0, nlev, 12)
    return np.concatenate([x1, x2]), np.concatenate([w1, w2])


def G_off_stable(x, y, mode):
    """G(x, y) for y on the unit sphere, eqs. Gextoffsurface / Gintoffsurface rewritten
    through d = |x - y| and r = |x| alone, which keeps them accurate as x approaches y.
    With x.y = (r^2 + 1 - d^2)/2:
      r - x.y = (d^2 - (r - 1)^2)/2 = (d - r + 1)(d + r - 1)/2,
      1 - x.y + d = ((d + 1)^2 - r^2)/2 = (d + 1 - r)(d + 1 + r)/2, so
      exterior: G_E = 2/d + log((d + r - 1)/(d + r + 1)),
      interior: G_I = 2/d + log(4/((d + 1 - r)(d + 1 + r)))."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    diff = x - y
    d = np.sqrt(np.sum(diff * diff, axis=-1))
    r = np.sqrt(np.sum(x * x, axis=-1))
    if mode == EXTERIOR:
        return 2.0 / d + np.log((d + (r - 1.0)) / (d + r + 1.0))
    return 2.0 / d + np.log(4.0 / ((d + (1.0 - r)) * (d + 1.0 + r)))


def near_potential(pre, c, fhat_j, x):
    """S sigma_j(x) for the patch centred at c with coefficients fhat_j, by direct
    quadrature of the off-surface Green's function against the density."""
    op = pre.op
    rad = op.rad
    x = np.asarray(x, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    t0, th0, r = _target_local(c, x)
    # distance of the target from the sphere, the near-singular scale of the integrand
    delta = abs(r - 1.0)
    blist = zernike.basis_list(pre.K)
    mk = np.array([m for _, m, _ in blist], dtype=np.float64)
    is_sin = np.array([cs == 1 for _, _, cs in blist])
    total = 0.0
    for pj in range(rad.npan):
        # the panel's rule graded toward t0 (split there when t0 lies inside the panel)
        tq, W, L = _panel_rule(rad, pj, t0)
        bq = L @ op.beta[pj * rad.nord:(pj + 1) * rad.nord, :]     # beta_k(t_q), nq x K
        cq = W[:, None] * bq * fhat_j[None, :]                       # nq x K
        for q in range(tq.size):
            th, wth = _theta_rule(th0, tq[q], t0, delta)
            y = local_to_global(c, np.full(th.size, tq[q]), th)
            g = G_off_stable(x[None, :], y, pre.mode) * wth
            ang = np.outer(th, mk)
            trig = np.where(is_sin[None, :], np.sin(ang), np.cos(ang))  # n_theta x K
            total += (g @ trig) @ cq[q]
    return float(total)


def potential(pre, centres, fhat, targets, near=2.5):
    """u(x) = sum_j S sigma_j(x) at (M, 3) targets: patches within near * eps (geodesic, from
    the target's radial projection) by near_potential, the others by their fine grids."""
    centres = np.asarray(centres, dtype=np.float64)
    targets = np.atleast_2d(np.asarray(targets, dtype=np.float64))
    N, K = centres.shape[0], pre.K
    F = np.asarray(fhat, dtype=np.float64).reshape(N, K)
    fine = patch_points(centres, pre.op.t_f, pre.op.th_f)           # N x nf x 3
    strength = pre.op.w[None, :] * (F @ pre.op.B.T)                   # N x nf
    out = np.zeros(targets.shape[0])
    for m, x in enumerate(targets):
        u = x / np.sqrt(x @ x)
        dist = np.arctan2(np.linalg.norm(np.cross(centres, u), axis=1), centres @ u)
        for j in range(N):
            if dist[j] < near * pre.eps:
                out[m] += near_potential(pre, centres[j], F[j], x)
            else:
                out[m] += G_off_surface(x[None, :], fine[j], pre.mode) @ strength[j]
    return out


def mean_field_outputs(pre, centres, fhat, targets):
    """The plotted fields (Section 2.2, eq. vtilde): exterior ubar = 1 - u, interior
    vbar = (v - 1)/(3 D) + (1 - |x|^2)/6 with D = -I_sigma."""
    targets = np.atleast_2d(np.asarray(targets, dtype=np.float64))
    u = potential(pre, centres, fhat, targets)
    if pre.mode == EXTERIOR:
        return 1.0 - u
    N = np.asarray(centres).shape[0]
    Is = pre.op.I @ np.asarray(fhat, dtype=np.float64).reshape(N, pre.K).sum(axis=0)
    return (u - 1.0) / (3.0 * (-Is)) + (1.0 - np.sum(targets * targets, axis=1)) / 6.0
