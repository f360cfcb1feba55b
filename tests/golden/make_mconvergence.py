"""Writes mconvergence_oracle.txt: the convergence study of Section 9.1 computed by the
oracle alone (N = 10 random patches, area fraction f = 0.05, interior, 13 x 20 panels,
ID and GMRES at 1e-15; reference M = 17 on 19 panels of 30 nodes). For each Zernike degree
M: K, the mean first passage time mu (eq. mufromsigma2) and the relative L2 residual on
patch 3 (eq. l2res). About 5 minutes on 8 cores.

    python tests/golden/make_mconvergence.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import operator as O, residual as R, solve as S  # noqa: E402
from paper_1906_04209_gb300 import layouts as L  # noqa: E402

N, F, SEED, PATCH = 10, 0.05, 1010, 3
CASES = [(M, 13, 20) for M in (3, 5, 7, 9, 11, 13, 15)] + [(17, 19, 30)]


def main():
    eps = L.eps_from_area_fraction(F, N)
    c = L.uniform(N, eps, L.rng(SEED))
    lines = ["# Oracle-only convergence study (Section 9.1): N = 10 uniform patches (layouts.uniform,",
             "# layouts.rng(1010)), f = 0.05, eps = 2 sqrt(f/N), interior, ID and GMRES at 1e-15.",
             "# Written by tests/golden/make_mconvergence.py from oracle/ only.",
             "# M K npan nord mu residual_patch3"]
    for M, npan, nord in CASES:
        K = (M + 1) * (M + 2) // 2
        pre = O.make_precompute(eps, 1, K, npan=npan, nord=nord, tau=1e-15)
        x, _, _, _ = S.gmres(lambda v: O.id_matvec(pre, c, v), O.rhs(pre, N), 1e-15)
        mu = S.outputs(pre.op.I, x, N, 1)[1]
        res = R.patch_residual(pre, c, x, PATCH)
        lines.append(f"{M} {K} {npan} {nord} {mu:.17g} {res:.6e}")
        print(lines[-1], flush=True)
    with open(os.path.join(HERE, "mconvergence_oracle.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
