"""CPU oracle for the 2D sweeping preconditioner (Engquist & Ying, Section 2).

TEST INFRASTRUCTURE ONLY.  Plain, slow, complex128 NumPy/SciPy code written from
the paper.  Only `tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` /
`--impl reference` legs of `bench.py` may import it.  It shares no code with the
CUDA path (`paper_1007_4290_gb300/`), and the CUDA path never imports it.

Modules
  assemble     O1: PML stretching (Eq. sigma) and the 5-point matrix A (Eq. helmd)
  direct       O2: direct solves of A u = f (banded LU, sparse LU)
  sweep_exact  O3: exact sweeping factorisation, Algorithms 2.1 / 2.2
  hmatrix      O4: weakly admissible H-matrix algebra (Section 2.3)
  hmatrix_strong O4s: strongly admissible H-matrix algebra with the randomized SVD
               for F = H . H (Section 2.3, the strongly admissible case)
  sweep_h      O4: approximate sweeping factorisation, Algorithms 2.5 / 2.6
  gmres        left-preconditioned GMRES on M A u = M f (Section 2.4)
  adjoint      misfit and its adjoint gradient with respect to c(x)

Parity pins live in tests/test_oracle_*.py.  Every function there is pinned
against something other than itself (closed forms, brute force, invariants).
"""
