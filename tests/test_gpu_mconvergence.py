"""The convergence study of Section 9.1 through the library: N = 10 random patches (area
fraction f = 0.05, interior), the library's own precompute (modal solve and ID on the
device) and FP64 solve for Zernike degrees M = 3, 5, ..., 15 and the refined reference
M = 17 on 19 panels of 30 nodes. Against the same study run by the oracle alone
(tests/golden/mconvergence_oracle.txt, written by make_mconvergence.py beside it):
  * at every M the library's mean first passage time equals the oracle's (the same
    discretisation; only the two IDs' skeletons differ, at the 1e-15 ID tolerance);
  * the relative L2 residual on a random patch (eq. l2res) agrees with the oracle's and
    decays spectrally in M, and the error of mu against the reference follows it down to
    the one-patch discretisation floor, as the paper reports."""
import os

import numpy as np
import pytest

from oracle.kernels import INTERIOR
from paper_1906_04209_gb300 import layouts as L, ncs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _cuda(libncs):
    assert torch.cuda.is_available(), "GPU test without a GPU"
    torch.cuda.set_device(0)


def _golden():
    rows = []
    for line in open(os.path.join(HERE, "golden", "mconvergence_oracle.txt")):
        if line.startswith("#") or not line.strip():
            continue
        M, K, npan, nord, mu, res = line.split()
        rows.append((int(M), int(K), int(npan), int(nord), float(mu), float(res)))
    return rows


def test_library_convergence_in_M_matches_oracle_study():
    N, f, seed, patch = 10, 0.05, 1010, 3
    eps = L.eps_from_area_fraction(f, N)
    c = L.uniform(N, eps, L.rng(seed))
    rows = []
    for M, K, npan, nord, mu_or, res_or in _golden():
        ctx = ncs.Context(eps, INTERIOR, K, npan=npan, nord=nord, id_tol=1e-15, method=ncs.METHOD_DIRECT)
        ctx.set_patches(c)
        r = ctx.solve(tol=1e-14, precision=ncs.FP64)
        res = ctx.patch_residual(patch, r["fhat"])
        rows.append((M, r["scalar"], res, mu_or, res_or, r["iterations"]))
    mu_ref = rows[-1][1]
    print("\nM   mu (library)        mu (oracle)         |mu - mu_ref|/mu_ref  residual (lib / oracle)")
    errs, res = [], []
    for M, mu, rs, mu_or, res_or, it in rows:
        e = abs(mu - mu_ref) / mu_ref
        print(f"{M:<3d} {mu:.15f}  {mu_or:.15f}  {e:.2e}            {rs:.2e} / {res_or:.2e}  ({it} products)")
        # the same discretised system as the oracle's study
        assert abs(mu - mu_or) <= 1e-11 * mu_or, (M, mu, mu_or)
        assert abs(rs - res_or) <= 1e-3 * res_or + 1e-13, (M, rs, res_or)
        if M < 17:
            errs.append(e)
            res.append(rs)
    assert all(b < a for a, b in zip(res[:5], res[1:6]))
    assert res[-1] < 1e-12 and errs[-1] < 1e-10
    assert all(e <= 2.0 * r for e, r in zip(errs[:4], res[:4]))
