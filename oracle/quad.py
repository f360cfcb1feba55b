"""Gauss rules and dyadically graded composite Gauss-Legendre rules.

Test infrastructure only (see the package docstring).
"""
import numpy as np
from scipy.special import roots_jacobi, roots_legendre


def gauss_legendre(a, b, n):
    """n-point Gauss-Legendre nodes and weights on [a, b]."""
    x, w = roots_legendre(n)
    return 0.5 * (a + b) + 0.5 * (b - a) * x, 0.5 * (b - a) * w


def gauss_jacobi_right(a, b, n):
    """Nodes/weights on [a, b] for integrals of phi(t) (b - t)^(-1/2) dt:
    Gauss-Jacobi with alpha = -1/2 at the right end, beta = 0 (Section 8.2)."""
    x, w = roots_jacobi(n, -0.5, 0.0)
    h = b - a
    t = a + 0.5 * (x + 1.0) * h
    # (b - t)^(-1/2) = (2/h)^(1/2) (1 - x)^(-1/2), dt = h/2 dx
    return t, w * np.sqrt(0.5 * h)


def graded_toward(a, b, s, nlev, n, hmax=None):
    """Composite n-point Gauss-Legendre rule on [a, b] with nlev dyadic levels of
    refinement toward the endpoint s (s == a or s == b); pieces longer than hmax
    (if given) are split into equal parts."""
    L = b - a
    edges = [0.0] + [L * 2.0 ** (-k) for k in range(nlev, 0, -1)] + [L]
    if hmax is not None:
        fine = [edges[0]]
        for u0, u1 in zip(edges[:-1], edges[1:]):
            k = int(np.ceil((u1 - u0) / hmax))
            fine.extend(u0 + (u1 - u0) * np.arange(1, k + 1) / k)
        edges = fine
    xs, ws = [], []
    for u0, u1 in zip(edges[:-1], edges[1:]):
        if s == a:
            x, w = gauss_legendre(a + u0, a + u1, n)
        else:
            x, w = gauss_legendre(b - u1, b - u0, n)
        xs.append(x)
        ws.append(w)
    return np.concatenate(xs), np.concatenate(ws)


def near_singular_rule(a, b, s, n_far=20, n_grad=10, nlev_sing=40, hmin=None):
    """A rule on [a, b] for an integrand analytic on [a, b] except for a
    singularity at the real point s (log-type if s is inside, nearby if outside).

    * s strictly inside: split at s, grade toward s with up to nlev_sing levels each
      side, stopping before a piece gets shorter than hmin (default 2e-13 max|a,b,s|)
      so that no node rounds onto s.
    * s outside at distance delta >= b - a: plain n_far-point Gauss-Legendre.
    * s outside closer than b - a: grade toward the nearer endpoint until the
      smallest interval is no longer than delta.
    """
    if a < s < b:
        floor = hmin if hmin is not None else 2e-13 * max(abs(a), abs(b), abs(s))
        n1 = int(min(nlev_sing, max(1, np.floor(np.log2((s - a) / floor)))))
        n2 = int(min(nlev_sing, max(1, np.floor(np.log2((b - s) / floor)))))
        x1, w1 = graded_toward(a, s, s, n1, n_grad)
        x2, w2 = graded_toward(s, b, s, n2, n_grad)
        return np.concatenate([x1, x2]), np.concatenate([w1, w2])
    delta = a - s if s <= a else s - b
    L = b - a
    if delta >= L:
        return gauss_legendre(a, b, n_far)
    if delta <= 0.0:
        nlev = nlev_sing
    else:
        nlev = int(np.ceil(np.log2(L / delta))) + 1
    end = a if s <= a else b
    return graded_toward(a, b, end, nlev, n_grad)


def barycentric_weights(x):
    """Barycentric weights for Lagrange interpolation on nodes x."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    w = np.ones(n)
    for j in range(n):
        d = x[j] - np.delete(x, j)
        w[j] = 1.0 / np.prod(d)
    return w


def lagrange_matrix(nodes, pts):
    """L[q, k] = k-th Lagrange cardinal polynomial on `nodes` evaluated at pts[q]."""
    nodes = np.asarray(nodes, dtype=np.float64)
    pts = np.asarray(pts, dtype=np.float64)
    n = nodes.size
    out = np.empty((pts.size, n))
    for k in range(n):
        others = np.delete(nodes, k)
        num = np.prod(pts[:, None] - others[None, :], axis=1)
        den = np.prod(nodes[k] - others)
        out[:, k] = num / den
    return out
