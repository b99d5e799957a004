"""O2: direct solves of the discrete system A u = f (Section 2.1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

With the row-by-row ordering A is banded with lower and upper bandwidth n.
`solve_banded_lu` factors it by banded LU with partial pivoting (LAPACK gbsv via
scipy.linalg.solve_banded); `SparseLU` uses SuperLU (scipy.sparse.linalg.splu)
and is the scalable variant for n >= 255.  Both compute the plain definition
u = A^{-1} f; the tests cross-check them.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla


def solve_banded_lu(disc, f):
    """u = A^{-1} f by banded LU with partial pivoting.  f: (N,) or (N, k)."""
    A = disc.matrix().tocoo()
    n, N = disc.n, disc.N
    ab = np.zeros((2 * n + 1, N), dtype=np.complex128)
    # LAPACK band storage: ab[n + i - j, j] = A[i, j]
    ab[n + A.row - A.col, A.col] = A.data
    return sla.solve_banded((n, n), ab, np.asarray(f, dtype=np.complex128))


class SparseLU:
    """Sparse LU of A (SuperLU with its default column ordering)."""

    def __init__(self, disc):
        self.lu = spla.splu(disc.matrix().tocsc())

    def solve(self, f, trans="N"):
        return self.lu.solve(np.asarray(f, dtype=np.complex128), trans=trans)
