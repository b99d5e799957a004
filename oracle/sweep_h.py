"""O4: approximate sweeping factorisation in H-matrix form, Algorithms 2.5 and 2.6.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Algorithm 2.5:  S~_1 = A_{1,1},  T~_1 = hinv(S~_1);
                S~_m = hsub(A_{m,m}, hdiagmul(A_{m,m-1}, hdiagmul(T~_{m-1}, A_{m-1,m}))),
                T~_m = hinv(S~_m).
Algorithm 2.6:  forward  u_{m+1} -= A_{m+1,m} hmatvec(T~_m, u_m)
                middle   u_m = hmatvec(T~_m, u_m)
                backward u_m -= hmatvec(T~_m, A_{m,m+1} u_{m+1})
The middle-loop product equals the forward-loop one (u_m is unchanged in
between), so it is evaluated once (the remark after Algorithm 2.2).
"""
import numpy as np
from . import hmatrix_strong as hs
from .hmatrix import HMatrix, Trunc, hinv, hsub, tree_depth


def tridiag_H(diag, off, lo, depth, L):
    """Exact H form of the tridiagonal block A_{m,m} restricted to [lo, hi): the
    off-diagonal blocks of a tridiagonal matrix are rank one (a single corner
    entry), the leaves are dense tridiagonal pieces."""
    n = diag.shape[0]
    H = HMatrix(lo, lo + n, depth, L)
    if depth == L:
        D = np.diag(diag).astype(complex)
        if n > 1:
            D[np.arange(n - 1), np.arange(1, n)] = off
            D[np.arange(1, n), np.arange(n - 1)] = off
        H.D = D
        return H
    k = (n + 1) // 2
    a = off[k - 1]                 # coupling between local index k-1 and k
    H.c11 = tridiag_H(diag[:k], off[:k - 1], lo, depth + 1, L)
    H.c22 = tridiag_H(diag[k:], off[k:], lo + k, depth + 1, L)
    e_last = np.zeros((k, 1), complex); e_last[-1, 0] = 1.0
    e_first = np.zeros((n - k, 1), complex); e_first[0, 0] = 1.0
    H.U12, H.V12 = a * e_last, e_first
    H.U21, H.V21 = a * e_first, e_last
    return H


class HSweep:
    """The approximate sweeping factorisation {T~_m} of A (Algorithm 2.5).

    admissibility "weak" (oracle.hmatrix) or "strong" (oracle.hmatrix_strong, whose
    F = H . H products draw Gaussian test vectors from numpy's generator seeded with
    `seed`)."""

    def __init__(self, disc, eps, leaf=8, rmax=None, admissibility="weak", seed=0):
        self.disc = disc
        self.tr = Trunc(eps, rmax)
        n = disc.n
        self.L = tree_depth(n, leaf)
        self.T = []
        if admissibility == "strong":
            self._setup_strong(leaf, seed)
            return
        assert admissibility == "weak"
        for m in range(n):
            Amm = tridiag_H(disc.diag[m], disc.east[m, 1:-1], 0, 0, self.L)
            if m == 0:
                S = Amm
            else:
                D = disc.A_off(m)          # A_{m,m-1} = A_{m-1,m}
                S = hsub(Amm, self.T[m - 1].diagmul(dl=D, dr=D), self.tr)
            self.T.append(hinv(S, self.tr))

    def _setup_strong(self, leaf, seed):
        """Algorithm 2.5 with strongly admissible H-matrices."""
        disc, n = self.disc, self.disc.n
        ct = hs.Clusters(n, leaf)
        rng = np.random.default_rng(seed)
        for m in range(n):
            S = hs.tridiag(ct, disc.diag[m], disc.east[m, 1:-1])
            if m > 0:
                D = disc.A_off(m)
                S = hs.hsub(S, self.T[m - 1].root.diagmul(D, D), self.tr)
            self.T.append(hs.StrongH(hs.hinv(S, self.tr, rng)))

    def apply(self, f):
        """Algorithm 2.6: u = M f.  f: (N,) or (N, k)."""
        disc, n = self.disc, self.disc.n
        f = np.asarray(f, dtype=complex)
        vec = f.ndim == 1
        u = f.reshape((n, n) + (() if vec else (f.shape[1],))).copy()
        w = np.empty_like(u)
        for m in range(n - 1):
            w[m] = self.T[m].matvec(u[m])
            D = disc.A_off(m + 1)
            u[m + 1] = u[m + 1] - (D if vec else D[:, None]) * w[m]
        w[n - 1] = self.T[n - 1].matvec(u[n - 1])
        u = w
        for m in range(n - 2, -1, -1):
            D = disc.A_off(m + 1)
            u[m] = u[m] - self.T[m].matvec((D if vec else D[:, None]) * u[m + 1])
        return u.reshape(f.shape)

    def ranks(self, m):
        """Ranks of the factorised blocks of T~_m, as {depth: [ranks]}."""
        out = {}
        for d, _, _, U, _ in self.T[m].blocks():
            out.setdefault(d, []).append(U.shape[1])
        return out
