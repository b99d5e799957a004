"""O4: hierarchical (H-) matrices on one layer, weakly admissible case (Section 2.3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Cluster tree (Section 2.3): the index set of a layer is bisected level by level;
a node [lo, hi) of size s has children [lo, lo + ceil(s/2)) and [lo + ceil(s/2), hi).
The paper assumes n = 2^k; for other n the ceil split is the reading taken.  All
leaves sit at the same depth L, the smallest L with ceil(n / 2^L) <= leaf.

Representation (weak admissibility: siblings are each other's interaction list):
a non-leaf node holds its two children (diagonal blocks, recursively) and the two
off-diagonal blocks in factorised form G12 = U12 V12^t, G21 = U21 V21^t; a leaf
holds its dense block.  Transposes are plain (not conjugate) transposes.

Truncation (recompression of a sum of low-rank terms, "Matrix addition"): QR of
the stacked left factors and of the stacked right factors, SVD of the small
product of the two R factors, keep sigma_k > eps * sigma_1 (at most rmax terms).
eps = 0 keeps every nonzero singular value, i.e. no approximation.
"""
import numpy as np


class Trunc:
    """Truncation rule: relative threshold eps and optional rank cap rmax."""

    def __init__(self, eps=0.0, rmax=None):
        self.eps = float(eps)
        self.rmax = rmax


def tree_depth(n, leaf):
    L = 0
    while -(-n // (1 << L)) > leaf:
        L += 1
    return L


def recompress(U, V, tr):
    """Truncated factorisation of U V^t: returns (U', V') with U' V'^t ~ U V^t."""
    n1, n2 = U.shape[0], V.shape[0]
    if U.shape[1] == 0:
        return U, V
    Q1, R1 = np.linalg.qr(U)
    Q2, R2 = np.linalg.qr(V)
    P, s, Wh = np.linalg.svd(R1 @ R2.T)
    if s.size == 0 or s[0] == 0.0:
        return np.zeros((n1, 0), complex), np.zeros((n2, 0), complex)
    k = int(np.count_nonzero(s > tr.eps * s[0]))
    if tr.rmax is not None:
        k = min(k, tr.rmax)
    return (Q1 @ P[:, :k]) * s[:k], Q2 @ Wh[:k, :].T


def svd_truncate_dense(B, tr):
    """Truncated SVD factorisation B ~ U V^t of a dense block."""
    if min(B.shape) == 0:
        return np.zeros((B.shape[0], 0), complex), np.zeros((B.shape[1], 0), complex)
    P, s, Wh = np.linalg.svd(B, full_matrices=False)
    if s[0] == 0.0:
        return np.zeros((B.shape[0], 0), complex), np.zeros((B.shape[1], 0), complex)
    k = int(np.count_nonzero(s > tr.eps * s[0]))
    if tr.rmax is not None:
        k = min(k, tr.rmax)
    return P[:, :k] * s[:k], Wh[:k, :].T


class HMatrix:
    """An H-matrix on the index range [lo, hi) of one layer."""

    def __init__(self, lo, hi, depth, L):
        self.lo, self.hi, self.depth, self.L = lo, hi, depth, L
        self.D = None
        self.c11 = self.c22 = None
        self.U12 = self.V12 = self.U21 = self.V21 = None

    # --- structure -------------------------------------------------------------
    @property
    def n(self):
        return self.hi - self.lo

    @property
    def is_leaf(self):
        return self.depth == self.L

    @property
    def split(self):
        return (self.n + 1) // 2

    def _shell(self):
        return HMatrix(self.lo, self.hi, self.depth, self.L)

    @staticmethod
    def from_dense(G, tr, leaf=8, lo=0, depth=0, L=None):
        """H-approximation of a dense matrix: off-diagonal blocks by truncated SVD."""
        n = G.shape[0]
        if L is None:
            L = tree_depth(n, leaf)
        H = HMatrix(lo, lo + n, depth, L)
        if depth == L:
            H.D = np.array(G, dtype=complex)
            return H
        k = H.split
        H.c11 = HMatrix.from_dense(G[:k, :k], tr, leaf, lo, depth + 1, L)
        H.c22 = HMatrix.from_dense(G[k:, k:], tr, leaf, lo + k, depth + 1, L)
        H.U12, H.V12 = svd_truncate_dense(G[:k, k:], tr)
        H.U21, H.V21 = svd_truncate_dense(G[k:, :k], tr)
        return H

    def to_dense(self):
        if self.is_leaf:
            return self.D.copy()
        k = self.split
        G = np.zeros((self.n, self.n), complex)
        G[:k, :k] = self.c11.to_dense()
        G[k:, k:] = self.c22.to_dense()
        G[:k, k:] = self.U12 @ self.V12.T
        G[k:, :k] = self.U21 @ self.V21.T
        return G

    def blocks(self):
        """Yield (depth, row range, col range, U, V) of every factorised block."""
        if self.is_leaf:
            return
        k = self.lo + self.split
        yield self.depth + 1, (self.lo, k), (k, self.hi), self.U12, self.V12
        yield self.depth + 1, (k, self.hi), (self.lo, k), self.U21, self.V21
        yield from self.c11.blocks()
        yield from self.c22.blocks()

    def leaves(self):
        if self.is_leaf:
            yield self
        else:
            yield from self.c11.leaves()
            yield from self.c22.leaves()

    # --- hmatvec ---------------------------------------------------------------
    def matvec(self, f):
        """hmatvec(G, f): G f by the 2 x 2 block recursion; f is (n,) or (n, k)."""
        if self.is_leaf:
            return self.D @ f
        k = self.split
        f1, f2 = f[:k], f[k:]
        y1 = self.c11.matvec(f1) + self.U12 @ (self.V12.T @ f2)
        y2 = self.U21 @ (self.V21.T @ f1) + self.c22.matvec(f2)
        return np.concatenate([y1, y2])

    def rmatvec(self, f):
        """G^t f (plain transpose)."""
        if self.is_leaf:
            return self.D.T @ f
        k = self.split
        f1, f2 = f[:k], f[k:]
        y1 = self.c11.rmatvec(f1) + self.V21 @ (self.U21.T @ f2)
        y2 = self.V12 @ (self.U12.T @ f1) + self.c22.rmatvec(f2)
        return np.concatenate([y1, y2])

    # --- hdiagmul --------------------------------------------------------------
    def diagmul(self, dl=None, dr=None):
        """hdiagmul: diag(dl) G diag(dr) (either may be None), by scaling the rows
        of the U factors / leaves with dl and of the V factors / leaves with dr."""
        H = self._shell()
        if self.is_leaf:
            D = self.D
            if dl is not None:
                D = dl[:, None] * D
            if dr is not None:
                D = D * dr[None, :]
            H.D = D
            return H
        k = self.split
        l1 = l2 = r1 = r2 = None
        if dl is not None:
            l1, l2 = dl[:k], dl[k:]
        if dr is not None:
            r1, r2 = dr[:k], dr[k:]
        H.c11 = self.c11.diagmul(l1, r1)
        H.c22 = self.c22.diagmul(l2, r2)
        H.U12 = self.U12 if l1 is None else l1[:, None] * self.U12
        H.V12 = self.V12 if r2 is None else r2[:, None] * self.V12
        H.U21 = self.U21 if l2 is None else l2[:, None] * self.U21
        H.V21 = self.V21 if r1 is None else r1[:, None] * self.V21
        return H

    def scale(self, a):
        H = self._shell()
        if self.is_leaf:
            H.D = a * self.D
            return H
        H.c11, H.c22 = self.c11.scale(a), self.c22.scale(a)
        H.U12, H.V12, H.U21, H.V21 = a * self.U12, self.V12, a * self.U21, self.V21
        return H


# --- hadd / hsub ------------------------------------------------------------------
def hadd(G, H, tr, alpha=1.0):
    """hadd(G, alpha H): blockwise sum; off-diagonal blocks stacked then recompressed."""
    R = G._shell()
    if G.is_leaf:
        R.D = G.D + alpha * H.D
        return R
    R.c11 = hadd(G.c11, H.c11, tr, alpha)
    R.c22 = hadd(G.c22, H.c22, tr, alpha)
    R.U12, R.V12 = recompress(np.hstack([G.U12, alpha * H.U12]), np.hstack([G.V12, H.V12]), tr)
    R.U21, R.V21 = recompress(np.hstack([G.U21, alpha * H.U21]), np.hstack([G.V21, H.V21]), tr)
    return R


def hsub(G, H, tr):
    """hsub(G, H) = hadd(G, -H)."""
    return hadd(G, H, tr, alpha=-1.0)


def add_lowrank(G, X, Y, tr):
    """G + X Y^t for an H-matrix G and a factorised term X Y^t, in H form."""
    R = G._shell()
    if G.is_leaf:
        R.D = G.D + X @ Y.T
        return R
    k = G.split
    X1, X2, Y1, Y2 = X[:k], X[k:], Y[:k], Y[k:]
    R.c11 = add_lowrank(G.c11, X1, Y1, tr)
    R.c22 = add_lowrank(G.c22, X2, Y2, tr)
    R.U12, R.V12 = recompress(np.hstack([G.U12, X1]), np.hstack([G.V12, Y2]), tr)
    R.U21, R.V21 = recompress(np.hstack([G.U21, X2]), np.hstack([G.V21, Y1]), tr)
    return R


# --- hmul ---------------------------------------------------------------------------
def hmul(G, H, tr):
    """hmul(G, H), weakly admissible case, by the 2 x 2 block product:
      (1,1) = G11 H11 + G12 H21   (recursion + a factorised term, then hadd)
      (1,2) = G11 H12 + G12 H22   (two factorised terms via hmatvec, recompressed)
      (2,1) = G21 H11 + G22 H21
      (2,2) = G21 H12 + G22 H22
    In G12 H21 = U12 (V12^t X21) Y21^t the middle product is formed first."""
    R = G._shell()
    if G.is_leaf:
        R.D = G.D @ H.D
        return R
    # G12 = U V^t, G21 = P Q^t ; H12 = X Y^t, H21 = Z W^t
    U, V, P, Q = G.U12, G.V12, G.U21, G.V21
    X, Y, Z, W = H.U12, H.V12, H.U21, H.V21
    R.c11 = add_lowrank(hmul(G.c11, H.c11, tr), U @ (V.T @ Z), W, tr)
    R.c22 = add_lowrank(hmul(G.c22, H.c22, tr), P @ (Q.T @ X), Y, tr)
    R.U12, R.V12 = recompress(np.hstack([G.c11.matvec(X), U]),
                              np.hstack([Y, H.c22.rmatvec(V)]), tr)
    R.U21, R.V21 = recompress(np.hstack([P, G.c22.matvec(Z)]),
                              np.hstack([H.c11.rmatvec(Q), W]), tr)
    return R


# --- hinv -------------------------------------------------------------------------
def hinv(G, tr):
    """hinv(G) by the 2 x 2 block inverse
        [[G11^-1 + G11^-1 G12 S^-1 G21 G11^-1, -G11^-1 G12 S^-1],
         [-S^-1 G21 G11^-1,                      S^-1          ]],
    S = G22 - G21 G11^-1 G12, with G11^-1 and S^-1 computed recursively and the
    leaf blocks inverted densely (LU with partial pivoting)."""
    R = G._shell()
    if G.is_leaf:
        R.D = np.linalg.inv(G.D)
        return R
    U, V = G.U12, G.V12            # G12 = U V^t
    P, Q = G.U21, G.V21            # G21 = P Q^t
    Ginv11 = hinv(G.c11, tr)
    # G21 G11^-1 G12 = P (Q^t G11^-1 U) V^t
    core = Q.T @ Ginv11.matvec(U)
    S = add_lowrank(G.c22, -P @ core, V, tr)
    Sinv = hinv(S, tr)
    A = Ginv11.matvec(U)           # G11^-1 U
    B = Ginv11.rmatvec(Q)          # (Q^t G11^-1)^t
    C = Sinv.rmatvec(V)            # (V^t S^-1)^t
    E = Sinv.matvec(P)             # S^-1 P
    # (1,2) = -G11^-1 U V^t S^-1 = -A C^t ; (2,1) = -S^-1 P Q^t G11^-1 = -E B^t
    R.U12, R.V12 = recompress(-A, C, tr)
    R.U21, R.V21 = recompress(-E, B, tr)
    # (1,1) = G11^-1 + A (V^t S^-1 P) B^t
    R.c11 = add_lowrank(Ginv11, A @ (V.T @ E), B, tr)
    R.c22 = Sinv
    return R
