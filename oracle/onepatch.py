"""The one-patch integral equation solver (Kaye & Greengard, Sections 5 and 8).

Test infrastructure only (see the package docstring).

Steps, in the paper's order:
  1. Fourier decomposition in theta reduces S sigma = f on a patch of radius eps
     to the modal equations 2 pi int_0^eps G_n(t, t') sigma_n(t') sin t' dt' = f_n(t)
     (eq. modalinteqn), with G_n(t, t') = (1/pi) int_0^pi G cos(n th) dth.
     The oracle evaluates G_n by brute quadrature of the full on-surface G
     (eqs. Gextonsurface / Gintonsurface) on a fixed theta-rule dyadically graded
     toward th = 0, so it never uses the G^(1), G^(2), G^(3) split (and so
     never meets the sign question in that split).
  2. sigma_n is discretised on m panels dyadically refined toward t = eps; a
     Legendre representation of order k on panels 1..m-1 and, on the last panel,
     sigma_n = g_n / sqrt(eps - t) with g_n a polynomial of degree k-1 (Gauss-Jacobi
     alpha = -1/2, beta = 0). Collocation at the quadrature nodes; entries by
     adaptive (graded) integration of G_n(t_i, .) against each basis function.
  3. One LU per mode; for each Zernike q_j with angular mode m_j the radial profile
     beta_j solves the mode-m_j system with right-hand side c_j R_{n_j}^{m_j}(t/eps),
     so b_j(t, theta) = beta_j(t) trig(m_j theta).
  4. Fine grid = radial collocation nodes x n_theta equispaced angles; weights =
     panel weight x sin t x 2 pi / n_theta (x sqrt(eps - t) on the Jacobi panel,
     because the stored unknown is sigma itself, not g). B(l, j) = b_j(x_l),
     I = w^T B (eq. getI).
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from . import zernike
from .kernels import G_on_surface
from .quad import (gauss_jacobi_right, gauss_legendre, graded_toward,
                   lagrange_matrix, near_singular_rule)

_THETA_RULE = {}


def theta_rule(nlev=50, n=10):
    """Composite Gauss-Legendre rule on [0, pi], dyadically graded toward 0, with no
    piece longer than pi/16 (so cos(n theta) is resolved for n up to ~20)."""
    key = (nlev, n)
    if key not in _THETA_RULE:
        _THETA_RULE[key] = graded_toward(0.0, np.pi, 0.0, nlev, n, hmax=np.pi / 16)
    return _THETA_RULE[key]


def chord_tt(t, tp, th):
    """|x - x'| for x = (t, th), x' = (t', 0) on the sphere:
    d^2 = 4 sin^2((t - t')/2) + 4 sin t sin t' sin^2(th/2) (rearranged from Section 8.1)."""
    A = 4.0 * np.sin(0.5 * (t - tp)) ** 2
    B = 4.0 * np.sin(t) * np.sin(tp)
    return np.sqrt(A[:, None] + B[:, None] * np.sin(0.5 * th)[None, :] ** 2)


def modal_kernels(t, tp, nmax, mode, chunk=4096):
    """G_n(t, t') for n = 0..nmax, by quadrature of (1/pi) int_0^pi G cos(n th) dth.
    t, tp: 1-D arrays of equal length. Returns (len, nmax+1)."""
    t = np.asarray(t, dtype=np.float64)
    tp = np.asarray(tp, dtype=np.float64)
    th, wth = theta_rule()
    C = np.cos(np.outer(th, np.arange(nmax + 1))) * (wth / np.pi)[:, None]
    out = np.empty((t.size, nmax + 1))
    for s in range(0, t.size, chunk):
        d = chord_tt(t[s:s + chunk], tp[s:s + chunk], th)
        out[s:s + chunk] = G_on_surface(d, mode) @ C
    return out


def modal_log_term(t, tp, nmax):
    """G_n^(2)(t, t') = (1/pi) int_0^pi log(2/|x-x'|) cos(n th) dth by the same
    quadrature (used to pin the quadrature against the paper's closed form)."""
    th, wth = theta_rule()
    C = np.cos(np.outer(th, np.arange(nmax + 1))) * (wth / np.pi)[:, None]
    d = chord_tt(np.asarray(t, float), np.asarray(tp, float), th)
    return np.log(2.0 / d) @ C


def modal_log_closed_form(t, tp, nmax):
    """The paper's closed form for G_n^(2) (Section 8.1):
    n = 0: -log(cos(t1/2) sin(t2/2)); n > 0: (tan(t1/2) cot(t2/2))^n / (2n),
    with t1 = min(t, t'), t2 = max(t, t')."""
    t1 = np.minimum(t, tp)
    t2 = np.maximum(t, tp)
    out = np.empty((np.size(t1), nmax + 1))
    out[:, 0] = -np.log(np.cos(0.5 * t1) * np.sin(0.5 * t2))
    ratio = np.tan(0.5 * t1) / np.tan(0.5 * t2)
    for n in range(1, nmax + 1):
        out[:, n] = ratio ** n / (2.0 * n)
    return out


@dataclass
class Radial:
    """Radial discretisation: panels, collocation nodes and weights."""
    eps: float
    npan: int
    nord: int
    edges: np.ndarray
    t: np.ndarray          # collocation nodes (npan*nord)
    wq: np.ndarray         # plain quadrature weights: int phi dt (Legendre panels),
                           # int phi (eps-t)^(-1/2) dt (Jacobi panel)
    w_sigma: np.ndarray    # weights for int g sigma dt with sigma stored pointwise
    panel: np.ndarray      # panel index of each node


def radial_discretisation(eps, npan=13, nord=20):
    """Panels [a_{j-1}, a_j], a_0 = 0, a_j = (1 - 2^-j) eps, a_m = eps (Section 8.2)."""
    edges = np.array([0.0] + [(1.0 - 2.0 ** (-j)) * eps for j in range(1, npan)] + [eps])
    ts, ws, wsig, pan = [], [], [], []
    for j in range(npan):
        a, b = edges[j], edges[j + 1]
        if j < npan - 1:
            x, w = gauss_legendre(a, b, nord)
            ws.append(w)
            wsig.append(w)
        else:
            x, w = gauss_jacobi_right(a, b, nord)
            ws.append(w)
            wsig.append(w * np.sqrt(eps - x))
        ts.append(x)
        pan.append(np.full(nord, j))
    return Radial(eps, npan, nord, edges, np.concatenate(ts), np.concatenate(ws),
                  np.concatenate(wsig), np.concatenate(pan))


def _panel_rule(rad, j, s):
    """Quadrature for int_{panel j} F(t') phi_k(t') sin t' dt' with a singularity of F
    at t' = s. Returns (t' nodes, weights incl. sin t' and the representation
    factor, basis matrix (nq x nord))."""
    a, b = rad.edges[j], rad.edges[j + 1]
    nodes = rad.t[j * rad.nord:(j + 1) * rad.nord]
    half = 0.5 * (b - a)
    mid = 0.5 * (a + b)
    if j < rad.npan - 1:
        tq, wq = near_singular_rule(a, b, s)
        L = lagrange_matrix((nodes - mid) / half, (tq - mid) / half)
        return tq, wq * np.sin(tq), L
    # Jacobi panel: sigma = g / sqrt(eps - t'), substitute t' = eps - u^2 so that
    # (eps - t')^(-1/2) dt' = 2 du on u in [0, sqrt(eps - a)].
    eps = rad.eps
    U = np.sqrt(eps - a)
    su = np.sqrt(max(eps - s, 0.0))
    # in u the singular point t' = s sits at u = su with dt'/du = -2u: keep the
    # innermost pieces long enough that t' stays >= ~30 ulp away from s
    hmin = max(2e-13 * U, 2e-13 * eps / su) if su > 0.0 else None
    uq, wu = near_singular_rule(0.0, U, su, hmin=hmin)
    tq = eps - uq * uq
    L = lagrange_matrix((nodes - mid) / half, (tq - mid) / half)
    L = L * np.sqrt(eps - nodes)[None, :]   # g(t_k) = sigma(t_k) sqrt(eps - t_k)
    return tq, 2.0 * wu * np.sin(tq), L


def collocation_matrices(rad, nmax, mode):
    """A_n[i, l] = 2 pi int G_n(t_i, t') phi_l(t') sin t' dt', n = 0..nmax, where
    phi_l is the cardinal basis of the piecewise representation (Section 8.2)."""
    nr = rad.t.size
    A = np.zeros((nmax + 1, nr, nr))
    for i in range(nr):
        ti = rad.t[i]
        tqs, wqs, Ls, cols = [], [], [], []
        for j in range(rad.npan):
            tq, wq, L = _panel_rule(rad, j, ti)
            tqs.append(tq)
            wqs.append(wq)
            Ls.append(L)
        tq = np.concatenate(tqs)
        Gn = modal_kernels(np.full(tq.size, ti), tq, nmax, mode)
        off = 0
        for j in range(rad.npan):
            nq = tqs[j].size
            blk = (Gn[off:off + nq] * wqs[j][:, None]).T @ Ls[j]   # (nmax+1) x nord
            A[:, i, j * rad.nord:(j + 1) * rad.nord] = 2.0 * np.pi * blk
            off += nq
    return A


def default_ntheta_fine(M):
    """Fine-grid azimuthal count (the paper leaves it open): M + 40 rounded up to
    an even number, so that a far-field target >= 2 eps away is integrated to
    ~2^-40 by the trapezoidal rule."""
    n = M + 40
    return n + (n % 2)


@dataclass
class OnePatch:
    eps: float
    mode: int
    K: int
    M: int
    rad: Radial
    ntheta: int
    beta: np.ndarray        # (nr, K) radial profiles
    B: np.ndarray           # (n_f, K)
    w: np.ndarray           # (n_f,)
    I: np.ndarray           # (K,)
    t_f: np.ndarray         # (n_f,) fine-grid t
    th_f: np.ndarray        # (n_f,) fine-grid theta
    A: np.ndarray = field(repr=False, default=None)  # collocation matrices


def solve_one_patch(eps, mode, K, npan=13, nord=20, ntheta=None, keep_A=False):
    """Precompute B, w, I for patch radius eps (Step 1 of Section 7)."""
    M = zernike.max_degree(K)
    rad = radial_discretisation(eps, npan, nord)
    mmax = max(m for _, m, _ in zernike.basis_list(K))
    A = collocation_matrices(rad, mmax, mode)
    lus = [sla.lu_factor(A[n]) for n in range(mmax + 1)]
    blist = zernike.basis_list(K)
    beta = np.empty((rad.t.size, K))
    for j, (n, m, c) in enumerate(blist):
        rhs = zernike.radial(n, m, rad.t / eps) / np.sqrt(zernike.norm2(n, m))
        beta[:, j] = sla.lu_solve(lus[m], rhs)
    nth = ntheta or default_ntheta_fine(M)
    th = 2.0 * np.pi * np.arange(nth) / nth
    t_f = np.repeat(rad.t, nth)
    th_f = np.tile(th, rad.t.size)
    trig = np.empty((th.size, K))
    for j, (n, m, c) in enumerate(blist):
        trig[:, j] = np.cos(m * th) if c == 0 else np.sin(m * th)
    B = (beta[:, None, :] * trig[None, :, :]).reshape(-1, K)
    w = np.repeat(rad.w_sigma * np.sin(rad.t), nth) * (2.0 * np.pi / nth)
    I = w @ B
    return OnePatch(eps, mode, K, M, rad, nth, beta, B, w, I, t_f, th_f,
                    A if keep_A else None)


def one_patch_residual(op, j, t_eval, th_eval):
    """Residual (S sigma_j - q_j) at independent points (t, theta) of the patch for
    sigma_j = b_j, evaluated through the same modal reduction; used for the
    eq. patcherrl2 check. Returns the residual values."""
    rad = op.rad
    n, m, c = zernike.basis_list(op.K)[j]
    vals = np.empty(t_eval.size)
    for q, (ti, thi) in enumerate(zip(t_eval, th_eval)):
        acc = 0.0
        for pj in range(rad.npan):
            tq, wq, L = _panel_rule(rad, pj, ti)
            Gm = modal_kernels(np.full(tq.size, ti), tq, m, op.mode)[:, m]
            coef = op.beta[pj * rad.nord:(pj + 1) * rad.nord, j]
            acc += 2.0 * np.pi * np.sum(wq * Gm * (L @ coef))
        trig = np.cos(m * thi) if c == 0 else np.sin(m * thi)
        target = zernike.radial(n, m, ti / op.eps) / np.sqrt(zernike.norm2(n, m))
        vals[q] = (acc - target) * trig
    return vals
