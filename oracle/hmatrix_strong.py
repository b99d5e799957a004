"""O4s: hierarchical (H-) matrices on one layer, strongly admissible case (Section 2.3,
the strongly admissible case; the randomized SVD for F = H . H).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Cluster tree: the same bisection as the weak case (oracle.hmatrix): a node [lo, hi) of
size s has children [lo, lo + ceil(s/2)) and [lo + ceil(s/2), hi); all leaves at depth L.
At depth l the 2^l nodes are numbered i = 0 .. 2^l - 1 from left to right.

Well-separatedness (strong): two clusters of one depth are well separated when the
distance between them is at least their width.  The clusters of one depth have equal
widths (up to one index when n is not a power of two), so clusters i and i' are well
separated exactly when at least one cluster lies between them: |i - i'| >= 2 (for
clusters of at least three indices; the index rule is the reading taken for all).  The
interaction list of i holds the i' that are well separated from i while their parents are
not, i.e. |i - i'| >= 2 and |floor(i/2) - floor(i'/2)| <= 1 (at most three entries).

A block (l, i, j) of an H-matrix (rows of cluster i, columns of cluster j, depth l) is
  'F'  factorised U V^t, when i and j are well separated,
  'D'  dense, at the leaf depth when they are not,
  'H'  split into its 2 x 2 children (l+1, 2i+a, 2j+b) otherwise,
so that near the diagonal the blocks are refined down to the dense leaves and their
neighbours.  The root block (0, 0, 0) is 'H' (or 'D' for a single leaf).

Operations (Section 2.3): hmatvec, hadd/hsub with recompression, hmul by the 2 x 2 block
product with every one of the eight forms of R = G . H (H hierarchical, F factorised), the
new form F = H . H by the randomized SVD of Halko, Martinsson and Tropp (K10), hinv by the
2 x 2 block inverse, hdiagmul.  Transposes are plain (not conjugate) transposes.
Truncation (oracle.hmatrix.Trunc): keep sigma_k > eps * sigma_1, at most rmax terms.
"""
import numpy as np

from .hmatrix import Trunc, recompress, svd_truncate_dense, tree_depth

# Extra Gaussian test vectors over the target rank in the randomized SVD; the paper does
# not state its oversampling, Halko, Martinsson and Tropp recommend 5 to 10.
RSVD_OVERSAMPLE = 8


class Clusters:
    """The bisection cluster tree of {0, ..., n-1} with leaves of at most `leaf` indices."""

    def __init__(self, n, leaf=8):
        self.n, self.leaf = n, leaf
        self.L = tree_depth(n, leaf)
        self.ranges = [[(0, n)]]
        for _ in range(self.L):
            nxt = []
            for lo, hi in self.ranges[-1]:
                k = lo + (hi - lo + 1) // 2
                nxt += [(lo, k), (k, hi)]
            self.ranges.append(nxt)

    def range(self, l, i):
        return self.ranges[l][i]

    def size(self, l, i):
        lo, hi = self.ranges[l][i]
        return hi - lo

    @staticmethod
    def well_separated(i, j):
        return abs(i - j) >= 2

    def kind(self, l, i, j):
        if self.well_separated(i, j):
            return "F"
        return "D" if l == self.L else "H"

    def interaction_list(self, l, i):
        """Clusters j of depth l in the interaction list of i."""
        if l == 0:
            return []
        p = i // 2
        out = []
        for q in (p - 1, p, p + 1):
            for j in (2 * q, 2 * q + 1):
                if 0 <= q < (1 << (l - 1)) and self.well_separated(i, j):
                    out.append(j)
        return out


class SBlock:
    """One block (l, i, j) of a strongly admissible H-matrix; `kind` is 'F', 'D' or 'H'.

    An 'F' block can stand for a block whose position would be refined (a low-rank
    operand restricted to a child position keeps its factorised form); the kind of a
    result is always the one its position prescribes (Clusters.kind)."""

    def __init__(self, ct, l, i, j, kind):
        self.ct, self.l, self.i, self.j, self.kind = ct, l, i, j, kind
        self.U = self.V = self.D = None
        self.ch = None                 # 2 x 2 list of children for 'H'

    @property
    def shape(self):
        return self.ct.size(self.l, self.i), self.ct.size(self.l, self.j)

    def _child_sizes(self):
        l, ct = self.l, self.ct
        rows = [ct.size(l + 1, 2 * self.i + a) for a in (0, 1)]
        cols = [ct.size(l + 1, 2 * self.j + b) for b in (0, 1)]
        return rows, cols

    def child(self, a, b):
        """The (a, b) child as an operand: an 'H' child, or the restriction of an 'F' block."""
        if self.kind == "H":
            return self.ch[a][b]
        assert self.kind == "F", "dense blocks have no children"
        rows, cols = self._child_sizes()
        r0 = 0 if a == 0 else rows[0]
        c0 = 0 if b == 0 else cols[0]
        C = SBlock(self.ct, self.l + 1, 2 * self.i + a, 2 * self.j + b, "F")
        C.U = self.U[r0:r0 + rows[a]]
        C.V = self.V[c0:c0 + cols[b]]
        return C

    # --- dense forms (for tests) ---------------------------------------------------
    def to_dense(self):
        m, p = self.shape
        if self.kind == "F":
            return self.U @ self.V.T
        if self.kind == "D":
            return self.D.copy()
        rows, cols = self._child_sizes()
        G = np.zeros((m, p), complex)
        for a in (0, 1):
            for b in (0, 1):
                r0 = 0 if a == 0 else rows[0]
                c0 = 0 if b == 0 else cols[0]
                G[r0:r0 + rows[a], c0:c0 + cols[b]] = self.ch[a][b].to_dense()
        return G

    def factor_blocks(self):
        """Yield every factorised block as (l, i, j, U, V)."""
        if self.kind == "F":
            yield self.l, self.i, self.j, self.U, self.V
        elif self.kind == "H":
            for a in (0, 1):
                for b in (0, 1):
                    yield from self.ch[a][b].factor_blocks()

    def dense_blocks(self):
        """Yield every dense block as (l, i, j, D)."""
        if self.kind == "D":
            yield self.l, self.i, self.j, self.D
        elif self.kind == "H":
            for a in (0, 1):
                for b in (0, 1):
                    yield from self.ch[a][b].dense_blocks()

    # --- hmatvec ---------------------------------------------------------------
    def matvec(self, f):
        """hmatvec: G f, by the 2 x 2 block recursion; f is (p,) or (p, k)."""
        if self.kind == "F":
            return self.U @ (self.V.T @ f)
        if self.kind == "D":
            return self.D @ f
        rows, cols = self._child_sizes()
        f0, f1 = f[:cols[0]], f[cols[0]:]
        y0 = self.ch[0][0].matvec(f0) + self.ch[0][1].matvec(f1)
        y1 = self.ch[1][0].matvec(f0) + self.ch[1][1].matvec(f1)
        return np.concatenate([y0, y1])

    def rmatvec(self, f):
        """G^t f (plain transpose)."""
        if self.kind == "F":
            return self.V @ (self.U.T @ f)
        if self.kind == "D":
            return self.D.T @ f
        rows, cols = self._child_sizes()
        f0, f1 = f[:rows[0]], f[rows[0]:]
        y0 = self.ch[0][0].rmatvec(f0) + self.ch[1][0].rmatvec(f1)
        y1 = self.ch[0][1].rmatvec(f0) + self.ch[1][1].rmatvec(f1)
        return np.concatenate([y0, y1])

    # --- hdiagmul ------------------------------------------------------------------
    def diagmul(self, dl=None, dr=None):
        """hdiagmul: diag(dl) G diag(dr) (either may be None)."""
        R = SBlock(self.ct, self.l, self.i, self.j, self.kind)
        if self.kind == "F":
            R.U = self.U if dl is None else dl[:, None] * self.U
            R.V = self.V if dr is None else dr[:, None] * self.V
            return R
        if self.kind == "D":
            D = self.D
            if dl is not None:
                D = dl[:, None] * D
            if dr is not None:
                D = D * dr[None, :]
            R.D = D
            return R
        rows, cols = self._child_sizes()
        dls = [None, None] if dl is None else [dl[:rows[0]], dl[rows[0]:]]
        drs = [None, None] if dr is None else [dr[:cols[0]], dr[cols[0]:]]
        R.ch = [[self.ch[a][b].diagmul(dls[a], drs[b]) for b in (0, 1)] for a in (0, 1)]
        return R

    def scale(self, alpha):
        R = SBlock(self.ct, self.l, self.i, self.j, self.kind)
        if self.kind == "F":
            R.U, R.V = alpha * self.U, self.V
        elif self.kind == "D":
            R.D = alpha * self.D
        else:
            R.ch = [[self.ch[a][b].scale(alpha) for b in (0, 1)] for a in (0, 1)]
        return R


# --- construction -------------------------------------------------------------------
def from_dense(ct, G, tr, l=0, i=0, j=0):
    """H-approximation of the dense block G at position (l, i, j): well-separated blocks by
    truncated SVD, the rest refined down to dense leaves."""
    B = SBlock(ct, l, i, j, ct.kind(l, i, j))
    if B.kind == "F":
        B.U, B.V = svd_truncate_dense(G, tr)
    elif B.kind == "D":
        B.D = np.array(G, dtype=complex)
    else:
        rows, cols = B._child_sizes()
        B.ch = [[from_dense(ct, G[(0 if a == 0 else rows[0]):(rows[0] if a == 0 else None),
                                  (0 if b == 0 else cols[0]):(cols[0] if b == 0 else None)],
                            tr, l + 1, 2 * i + a, 2 * j + b)
                 for b in (0, 1)] for a in (0, 1)]
    return B


def from_lowrank(ct, l, i, j, X, Y, tr):
    """The factorised term X Y^t written in the form of position (l, i, j)."""
    B = SBlock(ct, l, i, j, ct.kind(l, i, j))
    if B.kind == "F":
        B.U, B.V = recompress(X, Y, tr)
    elif B.kind == "D":
        B.D = X @ Y.T
    else:
        rows, cols = B._child_sizes()
        Xs = [X[:rows[0]], X[rows[0]:]]
        Ys = [Y[:cols[0]], Y[cols[0]:]]
        B.ch = [[from_lowrank(ct, l + 1, 2 * i + a, 2 * j + b, Xs[a], Ys[b], tr)
                 for b in (0, 1)] for a in (0, 1)]
    return B


def tridiag(ct, diag, off, l=0, i=0, j=0):
    """Exact strong H form of the symmetric tridiagonal matrix with diagonal `diag` and
    off-diagonal `off` (the block A_{m,m}): every entry couples neighbouring indices, which
    lie in the same or in adjacent clusters, so the well-separated blocks are zero (rank 0)
    and the band sits in the dense leaves."""
    B = SBlock(ct, l, i, j, ct.kind(l, i, j))
    if B.kind == "F":
        m, p = B.shape
        B.U, B.V = np.zeros((m, 0), complex), np.zeros((p, 0), complex)
    elif B.kind == "D":
        rlo, rhi = ct.range(l, i)
        clo, chi = ct.range(l, j)
        D = np.zeros((rhi - rlo, chi - clo), complex)
        for r in range(rlo, rhi):
            for c in (r - 1, r, r + 1):
                if clo <= c < chi:
                    D[r - rlo, c - clo] = diag[r] if c == r else off[min(r, c)]
        B.D = D
    else:
        B.ch = [[tridiag(ct, diag, off, l + 1, 2 * i + a, 2 * j + b) for b in (0, 1)]
                for a in (0, 1)]
    return B


def zeros(ct, l, i, j):
    m, p = ct.size(l, i), ct.size(l, j)
    return from_lowrank(ct, l, i, j, np.zeros((m, 0), complex), np.zeros((p, 0), complex),
                        Trunc())


# --- hadd / hsub ------------------------------------------------------------------------
def hadd(G, H, tr, alpha=1.0):
    """hadd(G, alpha H) for two blocks of the same position (its prescribed form): factorised
    blocks stacked and recompressed, dense blocks added, the rest blockwise."""
    ct, l, i, j = G.ct, G.l, G.i, G.j
    kind = ct.kind(l, i, j)
    if G.kind == "F" and H.kind == "F":
        X, Y = np.hstack([G.U, alpha * H.U]), np.hstack([G.V, H.V])
        return from_lowrank(ct, l, i, j, X, Y, tr)
    assert kind != "F", "a well-separated position holds factorised blocks only"
    R = SBlock(ct, l, i, j, kind)
    if kind == "D":
        R.D = G.to_dense() + alpha * H.to_dense()
        return R
    assert kind == "H"
    R.ch = [[hadd(G.child(a, b), H.child(a, b), tr, alpha) for b in (0, 1)] for a in (0, 1)]
    return R


def hsub(G, H, tr):
    return hadd(G, H, tr, alpha=-1.0)


# --- hmul ---------------------------------------------------------------------------------
def rsvd_product(G, H, tr, rng):
    """F = G . H for two hierarchical blocks, by the randomized SVD (K10): the range of
    G H is sampled with Gaussian test vectors, Y = G (H Omega) (two hmatvecs); Q is an
    orthonormal basis of Y; B = Q^* G H (Q^* the conjugate transpose) is formed as
    (H^t (G^t conj(Q)))^t; an SVD of the small B = P S W^t gives G H ~ (Q P S) W^t,
    truncated by `tr`.  The number of test vectors is
    rmax + RSVD_OVERSAMPLE (every column when no rank cap is set)."""
    m, p = G.shape[0], H.shape[1]
    k = min(m, p)
    if tr.rmax is not None:
        k = min(k, tr.rmax + RSVD_OVERSAMPLE)
    Om = rng.standard_normal((p, k)) + 1j * rng.standard_normal((p, k))
    Y = G.matvec(H.matvec(Om))
    Q, _ = np.linalg.qr(Y)
    Bt = H.rmatvec(G.rmatvec(Q.conj()))   # (Q^* G H)^t, p x k
    P, s, Wh = np.linalg.svd(Bt.T, full_matrices=False)
    if s.size == 0 or s[0] == 0.0:
        return np.zeros((m, 0), complex), np.zeros((p, 0), complex)
    r = int(np.count_nonzero(s > tr.eps * s[0]))
    if tr.rmax is not None:
        r = min(r, tr.rmax)
    return (Q @ P[:, :r]) * s[:r], Wh[:r, :].T


def hmul(G, H, tr, rng):
    """hmul(G, H) for G at (l, i, j) and H at (l, j, k); the result has the form of
    position (l, i, k).  The eight forms of R = G . H:
      any = F . any   ->  U (H^t V)^t           (F = F.H, F = F.F, H = F.H, H = F.F)
      any = H . F     ->  (G X) Y^t             (F = H.F, H = H.F)
      H = H . H       ->  2 x 2 block product, sums by hadd
      F = H . H       ->  randomized SVD (rsvd_product)
    a factorised product landing on an 'H' position is written in that form
    (from_lowrank); dense leaves multiply densely."""
    ct, l, i, k = G.ct, G.l, G.i, H.j
    kind = ct.kind(l, i, k)
    if G.kind == "F":
        return from_lowrank(ct, l, i, k, G.U, H.rmatvec(G.V), tr)
    if H.kind == "F":
        return from_lowrank(ct, l, i, k, G.matvec(H.U), H.V, tr)
    if G.kind == "D" or H.kind == "D":
        # leaf depth: both operands are dense blocks
        P = G.to_dense() @ H.to_dense()
        if kind == "F":
            R = SBlock(ct, l, i, k, "F")
            R.U, R.V = svd_truncate_dense(P, tr)
            return R
        R = SBlock(ct, l, i, k, "D")
        R.D = P
        return R
    if kind == "F":
        R = SBlock(ct, l, i, k, "F")
        R.U, R.V = rsvd_product(G, H, tr, rng)
        return R
    R = SBlock(ct, l, i, k, "H")
    R.ch = [[hadd(hmul(G.child(a, 0), H.child(0, b), tr, rng),
                  hmul(G.child(a, 1), H.child(1, b), tr, rng), tr)
             for b in (0, 1)] for a in (0, 1)]
    return R


# --- hinv ---------------------------------------------------------------------------------
def hinv(G, tr, rng):
    """hinv(G) for a diagonal block, by the 2 x 2 block inverse
        [[G11^-1 + G11^-1 G12 S^-1 G21 G11^-1, -G11^-1 G12 S^-1],
         [-S^-1 G21 G11^-1,                      S^-1          ]],
    S = G22 - G21 G11^-1 G12; G11^-1 and S^-1 recursively, dense leaves by LU with
    partial pivoting."""
    ct, l, i = G.ct, G.l, G.i
    R = SBlock(ct, l, i, i, G.kind)
    if G.kind == "D":
        R.D = np.linalg.inv(G.D)
        return R
    G11, G12, G21, G22 = G.child(0, 0), G.child(0, 1), G.child(1, 0), G.child(1, 1)
    X11 = hinv(G11, tr, rng)
    Z = hmul(G21, X11, tr, rng)                  # G21 G11^-1
    S = hsub(G22, hmul(Z, G12, tr, rng), tr)     # G22 - G21 G11^-1 G12
    X22 = hinv(S, tr, rng)                       # S^-1
    W = hmul(hmul(X11, G12, tr, rng), X22, tr, rng)   # G11^-1 G12 S^-1
    R.ch = [[hadd(X11, hmul(W, Z, tr, rng), tr), W.scale(-1.0)],
            [hmul(X22, Z, tr, rng).scale(-1.0), X22]]
    return R


class StrongH:
    """A strongly admissible H-matrix on one layer: the root block and its cluster tree."""

    def __init__(self, root):
        self.root, self.ct = root, root.ct

    def matvec(self, f):
        return self.root.matvec(f)

    def to_dense(self):
        return self.root.to_dense()

    def diagmul(self, dl=None, dr=None):
        return StrongH(self.root.diagmul(dl, dr))

    def blocks(self):
        """(depth, row range, col range, U, V) of every factorised block."""
        for l, i, j, U, V in self.root.factor_blocks():
            yield l, self.ct.range(l, i), self.ct.range(l, j), U, V
