"""The convergence study of Section 9.1 on the oracle: for N = 10 random patches (area
fraction f = 0.05, interior), the relative L2 residual on a random patch (eq. l2res) and the
self-consistent error of the mean first passage time against a refined run (M = 17, 19
panels of 30 nodes) as the Zernike degree M grows.

Test infrastructure only (see the package docstring). Run: python -m oracle.mconvergence
(about 5 minutes on 8 cores).
"""
import time

from . import operator as O
from . import residual as R
from . import solve as S


def study(N=10, f=0.05, seed=1010, patch=3, degrees=(3, 5, 7, 9, 11, 13, 15), ref=(17, 19, 30)):
    from paper_1906_04209_gb300 import layouts as L
    eps = L.eps_from_area_fraction(f, N)
    c = L.uniform(N, eps, L.rng(seed))
    rows = []
    for M, npan, nord in [(M, 13, 20) for M in degrees] + [ref]:
        t0 = time.time()
        pre = O.make_precompute(eps, 1, (M + 1) * (M + 2) // 2, npan=npan, nord=nord, tau=1e-15)
        x, it, _, _ = S.gmres(lambda v: O.id_matvec(pre, c, v), O.rhs(pre, N), 1e-15)
        mu = S.outputs(pre.op.I, x, N, 1)[1]
        rows.append((M, mu, R.patch_residual(pre, c, x, patch), it, time.time() - t0))
    mu_ref = rows[-1][1]
    return [(M, mu, abs(mu - mu_ref) / mu_ref, res, it, sec) for M, mu, res, it, sec in rows[:-1]], mu_ref


if __name__ == "__main__":
    out, mu_ref = study()
    print(f"reference mu = {mu_ref:.15f}")
    print("M   mu                  |mu - mu_ref|/mu_ref  residual   GMRES its")
    for M, mu, err, res, it, sec in out:
        print(f"{M:<3d} {mu:.15f}  {err:.2e}            {res:.2e}   {it}   ({sec:.0f} s)")
