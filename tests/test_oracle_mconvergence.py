"""The convergence study of Section 9.1 on the oracle: for N = 10 random patches (area
fraction f = 0.05, interior), the relative L2 residual on a random patch (eq. l2res) and the
self-consistent error of the mean first passage time against a refined run (M = 17, 19
panels of 30 nodes) as the Zernike degree M grows. About 5 minutes on 8 cores, so it runs
only when NCS_STUDY is set:  NCS_STUDY=1 python -m pytest tests/test_oracle_mconvergence.py -s
"""
import os
import time

import pytest

from oracle import operator as O, residual as R, solve as S
from paper_1906_04209_gb300 import layouts as L


@pytest.mark.slow
@pytest.mark.skipif(not os.environ.get("NCS_STUDY"), reason="study: set NCS_STUDY=1 to run")
def test_spectral_convergence_in_M():
    N, f, seed, patch = 10, 0.05, 1010, 3
    eps = L.eps_from_area_fraction(f, N)
    c = L.uniform(N, eps, L.rng(seed))
    rows = []
    for M, npan, nord in [(M, 13, 20) for M in (3, 5, 7, 9, 11, 13, 15)] + [(17, 19, 30)]:
        t0 = time.time()
        pre = O.make_precompute(eps, 1, (M + 1) * (M + 2) // 2, npan=npan, nord=nord, tau=1e-15)
        x, it, _, _ = S.gmres(lambda v: O.id_matvec(pre, c, v), O.rhs(pre, N), 1e-15)
        mu = S.outputs(pre.op.I, x, N, 1)[1]
        rows.append((M, mu, R.patch_residual(pre, c, x, patch), it, time.time() - t0))
    mu_ref = rows[-1][1]
    print(f"\nreference mu = {mu_ref:.15f}\nM   mu                  |mu - mu_ref|/mu_ref  residual   GMRES its")
    errs, res = [], []
    for M, mu, r, it, sec in rows[:-1]:
        errs.append(abs(mu - mu_ref) / mu_ref)
        res.append(r)
        print(f"{M:<3d} {mu:.15f}  {errs[-1]:.2e}            {r:.2e}   {it}   ({sec:.0f} s)")
    # spectral decay of the residual; the mu error follows it down to the one-patch floor
    assert all(b < a for a, b in zip(res[:5], res[1:6]))
    assert res[-1] < 1e-12 and errs[-1] < 1e-10
    assert all(e <= 2.0 * r for e, r in zip(errs[:4], res[:4]))
