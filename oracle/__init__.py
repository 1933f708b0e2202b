"""Plain, slow CPU FP64 oracle for the DG-SBM hp-multigrid / FGMRES path.

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only `tests/`, `__graft_entry__.smoke()` and
`bench.py`'s CPU-baseline / reference arm may import it.  The CUDA library and its
Python binding never import, link or call anything in here, and nothing in here
imports them: the two share no code, no tables and no constants.  The only shared
module is `workloads`, which produces seeded inputs and does none of the method's
arithmetic.

What it computes (paper sections / equations of arXiv 2506.12899):
  quadrature  Gauss-Legendre rules and the nodal Lagrange basis (Sec. 2.2, basis choice)
  geometry    level sets, volume fraction kappa (Eq. 4), active cells (Sec. 2.1),
              surrogate faces, closest-point shift vectors d (Eqs. 19-22, Sec. 4.2)
  dgsbm       the DG-SBM bilinear form a_h and right-hand side (Eqs. 7, 10, 11) assembled
              into a sparse matrix by explicit quadrature loops; the L2 error
  multigrid   the hp level hierarchy (Sec. 3), cell-wise block Gauss-Seidel as successive
              subspace correction (Eqs. 14, 16), prolongation/restriction (Eqs. 17, 18),
              the coarse direct solve and one V-cycle
  krylov      flexible GMRES(m), right-preconditioned, classical Gram-Schmidt twice

Every function names the passage it follows.  Where the paper is silent or ambiguous the
reading taken is stated in the function's docstring.
"""
