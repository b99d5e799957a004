"""O3: the exact sweeping factorisation, Algorithms 2.1 and 2.2 (Eq. Afact).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

S_1 = A_{1,1},  S_m = A_{m,m} - A_{m,m-1} S_{m-1}^{-1} A_{m-1,m},  T_m = S_m^{-1},
all dense n x n.  O(n^4) work: only for small n.
"""
import numpy as np


def setup_exact(disc):
    """Algorithm 2.1: returns the list [T_1, ..., T_n] (0-based list index m-1)."""
    n = disc.n
    T = []
    S = disc.A_mm(0)
    T.append(np.linalg.inv(S))
    for m in range(1, n):
        D = disc.A_off(m)                        # A_{m,m-1} = A_{m-1,m}, diagonal
        S = disc.A_mm(m) - (D[:, None] * T[m - 1]) * D[None, :]
        T.append(np.linalg.inv(S))
    return T


def solve_exact(disc, T, f):
    """Algorithm 2.2: u = A^{-1} f with the dense factors T_m.

    f: (N,) complex.  The products T_m u_m of the second and third loops are the
    same (u_m is not touched in between); the paper remarks that one evaluation
    suffices, so it is computed once and reused."""
    n = disc.n
    u = np.array(f, dtype=np.complex128).reshape(n, n).copy()     # u_m = f_m
    w = np.empty_like(u)
    for m in range(n - 1):                                         # forward loop
        w[m] = T[m] @ u[m]
        u[m + 1] = u[m + 1] - disc.A_off(m + 1) * w[m]
    w[n - 1] = T[n - 1] @ u[n - 1]
    u = w.copy()                                                   # middle loop
    for m in range(n - 2, -1, -1):                                 # backward loop
        u[m] = u[m] - T[m] @ (disc.A_off(m + 1) * u[m + 1])
    return u.ravel()
