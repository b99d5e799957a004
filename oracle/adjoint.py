"""Misfit J(c) = 1/2 sum_s ||R u_s - d_s||^2 with A(c) u_s = f_s, and its gradient.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Only the diagonal of A depends on c (Eq. helmd): dA_ii/dc_i = -2 omega^2 /
((s1 s2)_i c_i^3).  With A^H lambda_s = -R^t (R u_s - d_s),
  dJ/dc_i = sum_s Re( conj(lambda_{s,i}) (dA_ii/dc_i) u_{s,i} ).
The adjoint system is solved here with the conjugate-transposed sparse LU, by
the plain definition, not through the symmetry of A.
"""
import numpy as np
from .assemble import Discretization
from .direct import SparseLU


def misfit_and_gradient(c, omega, pml_width, F, rec_idx, d, C=2 * np.pi):
    """F: (nsrc, N) sources; rec_idx: receiver node indices; d: (nsrc, nrec).
    Returns (J, grad (n, n), U (nsrc, N))."""
    disc = Discretization(c, omega, pml_width, C)
    lu = SparseLU(disc)
    U = np.stack([lu.solve(f) for f in F])
    J = 0.0
    g = np.zeros(disc.N)
    dA = disc.d_diag_dc().ravel()
    for s in range(F.shape[0]):
        r = U[s, rec_idx] - d[s]
        J += 0.5 * np.vdot(r, r).real
        rhs = np.zeros(disc.N, complex)
        np.add.at(rhs, rec_idx, -r)
        lam = lu.solve(rhs, trans="H")
        g += (np.conj(lam) * dA * U[s]).real
    return J, g.reshape(disc.n, disc.n), U


def misfit(c, omega, pml_width, F, rec_idx, d, C=2 * np.pi):
    disc = Discretization(c, omega, pml_width, C)
    lu = SparseLU(disc)
    J = 0.0
    for s in range(F.shape[0]):
        r = lu.solve(F[s])[rec_idx] - d[s]
        J += 0.5 * np.vdot(r, r).real
    return J
