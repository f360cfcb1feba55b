"""FP64 CPU oracle for the narrow capture / narrow escape solver of Kaye &
Greengard (arXiv 1906.04209).

TEST INFRASTRUCTURE ONLY. Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package. The
product path (the CUDA library and its binding) never calls it, and this package
never imports the product path.

Every function is a plain, slow, step-by-step restatement of the paper:
  kernels.py   Green's functions on and off the sphere (Section 2.1)
  zernike.py   Zernike basis, sampling nodes and transform P (Section 4)
  quad.py      Gauss rules and dyadically graded composite rules
  onepatch.py  modal one-patch solver: B, fine grid, weights, I (Sections 5, 8)
  geometry.py  patch frames (local polar coordinates about each centre)
  idcomp.py    interpolative decomposition of the far field, T = Pi W B (Section 7.1)
  operator.py  dense operator, ID-direct matvec (eq. opinteqnsdisc, Section 7.1)
  solve.py     GMRES, dense LU, I_sigma -> mu / capacitance (Sections 2, 6)
  rows.c       plain-C FP64 ID-direct sums at sampled target nodes (large N)

Functions whose value no independent pin fixes say "parity unpinned" in their
docstring.
"""
