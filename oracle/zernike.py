"""Zernike basis on a patch, sampling nodes and the discrete Zernike transform P
(Kaye & Greengard, Section 4 and Section 6).

Test infrastructure only (see the package docstring).

Readings of the paper taken here:
  * The basis is the standard Zernike set: n - m even, cos(m theta) for m >= 0 and
    sin(m theta) for m > 0, normalised to unit L2 norm on the unit disk with the
    planar measure r dr dtheta (eq. zorthog). r is the arclength from the patch
    centre divided by eps.
  * Functions are ordered by n ascending, then |m| ascending, cos before sin, and
    the first K are kept. For K = (M+1)(M+2)/2 this is the paper's truncation
    0 <= m <= n <= M; K = 64 and 128 end on complete cos/sin pairs.
  * The sampling grid is Gauss-Legendre with M+1 nodes in r in [0, 1] times the
    trapezoidal rule with 2M+1 equispaced angles, so K* = (M+1)(2M+1); this
    integrates products of two basis functions exactly.
"""
import numpy as np
from scipy.special import eval_jacobi, roots_legendre


def basis_list(K):
    """List of (n, m, c) for the first K basis functions; c = 0 for cos, 1 for sin."""
    out = []
    n = 0
    while len(out) < K:
        for m in range(n % 2, n + 1, 2):
            out.append((n, m, 0))
            if m > 0:
                out.append((n, m, 1))
        n += 1
    return out[:K]


def max_degree(K):
    """M = the largest radial degree n among the first K basis functions."""
    return max(n for n, _, _ in basis_list(K))


def radial(n, m, r):
    """R_n^m(r) = (-1)^((n-m)/2) r^m P_{(n-m)/2}^{(m,0)}(1 - 2 r^2) (Section 4)."""
    k = (n - m) // 2
    r = np.asarray(r, dtype=np.float64)
    return (-1.0) ** k * r ** m * eval_jacobi(k, m, 0, 1.0 - 2.0 * r * r)


def norm2(n, m):
    """int_0^{2pi} int_0^1 Z^2 r dr dtheta = (1 + delta_{m0}) pi / (2n + 2) (eq. zorthog)."""
    return (2.0 if m == 0 else 1.0) * np.pi / (2.0 * n + 2.0)


def q_eval(K, r, theta):
    """Values of the orthonormal q_1..q_K at points (r, theta) on the unit disk.
    Returns an array of shape (len(r), K)."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    theta = np.atleast_1d(np.asarray(theta, dtype=np.float64))
    out = np.empty((r.size, K))
    for j, (n, m, c) in enumerate(basis_list(K)):
        trig = np.cos(m * theta) if c == 0 else np.sin(m * theta)
        out[:, j] = radial(n, m, r) * trig / np.sqrt(norm2(n, m))
    return out


def sampling_nodes(M):
    """Zernike sampling nodes (r_k, theta_b) on the unit disk, radial-major order,
    and the tensor-product weights w = w_GL(r) * r * 2 pi/(2M+1)."""
    x, wx = roots_legendre(M + 1)
    r = 0.5 * (x + 1.0)
    wr = 0.5 * wx
    nth = 2 * M + 1
    th = 2.0 * np.pi * np.arange(nth) / nth
    R, TH = np.meshgrid(r, th, indexing="ij")
    W = (wr * r)[:, None] * np.full(nth, 2.0 * np.pi / nth)[None, :]
    return R.ravel(), TH.ravel(), W.ravel()


def transform(K):
    """The discrete Zernike transform P (K x K*): P[j, k] = w_k q_j(x_k).
    Returns (P, r_nodes, theta_nodes)."""
    M = max_degree(K)
    r, th, w = sampling_nodes(M)
    Q = q_eval(K, r, th)  # K* x K
    return (Q * w[:, None]).T.copy(), r, th


def synthesis(K):
    """Q_z (K* x K): q_j sampled at the sampling nodes."""
    M = max_degree(K)
    r, th, _ = sampling_nodes(M)
    return q_eval(K, r, th)
