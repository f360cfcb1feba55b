"""GMRES, dense solve and the scalar outputs (Kaye & Greengard, Sections 2 and 6-7).

Test infrastructure only (see the package docstring).

Readings (the paper does not fix the GMRES details): x0 = 0, no restart,
modified Gram-Schmidt, stop when the estimated ||b - A x|| / ||b|| <= tol;
the true residual is recomputed at exit.
"""
import numpy as np
import scipy.linalg as sla

from .kernels import EXTERIOR


def gmres(matvec, b, tol=1e-10, maxit=200):
    """Returns (x, iterations, residual-estimate history, true relative residual)."""
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    n = b.size
    V = np.zeros((maxit + 1, n))
    H = np.zeros((maxit + 1, maxit))
    cs = np.zeros(maxit)
    sn = np.zeros(maxit)
    g = np.zeros(maxit + 1)
    g[0] = nb
    V[0] = b / nb
    hist = [1.0]
    k = 0
    for k in range(maxit):
        w = matvec(V[k])
        for j in range(k + 1):
            H[j, k] = w @ V[j]
            w = w - H[j, k] * V[j]
        H[k + 1, k] = np.linalg.norm(w)
        if H[k + 1, k] > 0:
            V[k + 1] = w / H[k + 1, k]
        for j in range(k):
            a, c = H[j, k], H[j + 1, k]
            H[j, k] = cs[j] * a + sn[j] * c
            H[j + 1, k] = -sn[j] * a + cs[j] * c
        r = np.hypot(H[k, k], H[k + 1, k])
        cs[k] = H[k, k] / r
        sn[k] = H[k + 1, k] / r
        H[k, k] = r
        H[k + 1, k] = 0.0
        g[k + 1] = -sn[k] * g[k]
        g[k] = cs[k] * g[k]
        hist.append(abs(g[k + 1]) / nb)
        if hist[-1] <= tol:
            break
    m = k + 1
    y = sla.solve_triangular(H[:m, :m], g[:m])
    x = V[:m].T @ y
    true = np.linalg.norm(b - matvec(x)) / nb
    return x, m, np.array(hist), true


def dense_solve(A, b):
    return sla.lu_solve(sla.lu_factor(A), b)


def outputs(I, fhat, N, mode):
    """I_sigma = I . sum_i f_i (eq. getI). Interior: mu = 1/(3 I_sigma) - 3/5
    (eq. mufromsigma2). Exterior: the capacitance C = 4 pi I_sigma (reading: the
    representation u = int G_E sigma with u = (1/4pi) int G_E du/dn gives
    sigma = (1/4pi) du/dn, so |J| = 4 pi I_sigma; J = -I_sigma as printed drops the
    4 pi). Returns (I_sigma, mu_or_C)."""
    F = np.asarray(fhat, dtype=np.float64).reshape(N, -1)
    Is = float(np.asarray(I) @ F.sum(axis=0))
    if mode == EXTERIOR:
        return Is, 4.0 * np.pi * Is
    return Is, 1.0 / (3.0 * Is) - 0.6
