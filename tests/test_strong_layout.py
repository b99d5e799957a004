"""Host logic of the strongly admissible GPU path (no device needed): the block plan the
kernels fill (hsweep_strong_plan) against the paper's interaction lists (Section 2.3, the
oracle's Clusters), the exactness of the expanded sibling-pair layout, and the Gaussian test
vectors of the randomized SVD (hsweep_rsvd_normals)."""
import numpy as np
import pytest

from oracle.hmatrix_strong import Clusters


@pytest.fixture(scope="module")
def hs():
    import os
    import __graft_entry__ as g
    b = g._build_module()
    if not os.path.exists(b.LIB):
        b.build()
    import paper_1007_4290_gb300 as m
    return m


@pytest.mark.parametrize("n,leaf,R", [(31, 8, 2), (127, 8, 2), (100, 8, 1), (1023, 8, 2), (64, 4, 3)])
def test_far_blocks_are_exactly_the_interaction_lists(hs, n, leaf, R):
    ct = Clusters(n, leaf)
    far, near, ranks = hs.strong_plan(n, leaf, R)
    got = set()
    for a, b, ru0, rw0, su, sw, col, l in far.tolist():
        assert b == a + 1 and a % 2 == 0
        la = a.bit_length() - 1
        assert la < l <= ct.L
        # locate the clusters of depth l by their rows
        alo = ct.range(la, a - (1 << la))[0]
        blo = ct.range(la, b - (1 << la))[0]
        i = [k for k in range(1 << l) if ct.range(l, k) == (alo + ru0, alo + ru0 + su)]
        j = [k for k in range(1 << l) if ct.range(l, k) == (blo + rw0, blo + rw0 + sw)]
        assert len(i) == 1 and len(j) == 1
        got.add((int(l), i[0], j[0]))
        assert 0 <= col and col + R <= ranks[a]
    want = {(l, i, j) for l in range(ct.L + 1) for i in range(1 << l)
            for j in ct.interaction_list(l, i) if j > i}
    assert got == want
    # the near field: one dense corner per sibling pair = every pair of neighbouring leaves
    corners = set()
    for a, b, ca0, na, nb, col in near.tolist():
        la = a.bit_length() - 1
        alo, ahi = ct.range(la, a - (1 << la))
        i = [k for k in range(1 << ct.L) if ct.range(ct.L, k) == (alo + ca0, alo + ca0 + na)]
        assert len(i) == 1 and ct.range(ct.L, i[0] + 1)[0] == ahi and ct.size(ct.L, i[0] + 1) == nb
        corners.add(i[0])
        assert ranks[a] == ranks[b] == col + nb == 3 * R * (ct.L - la) + nb
    assert corners == set(range((1 << ct.L) - 1))


@pytest.mark.parametrize("n,leaf,R", [(127, 8, 2), (45, 4, 1)])
def test_expanded_layout_represents_the_strong_matrix_exactly(hs, n, leaf, R):
    # a random strongly admissible symmetric matrix (rank-R far blocks, dense near field,
    # dense diagonal leaves) written into the sibling-pair factors by the plan's columns
    # reproduces itself: every block of every sibling pair is F_a F_b^t
    rng = np.random.default_rng(n)
    ct = Clusters(n, leaf)
    L = ct.L
    far, near, ranks = hs.strong_plan(n, leaf, R)
    ranks = ranks.tolist()
    T = np.zeros((n, n), complex)
    Fs = {}

    def rows(v):
        l = v.bit_length() - 1
        return ct.range(l, v - (1 << l))

    for v in range(2, 1 << (L + 1)):
        Fs[v] = np.zeros((rows(v)[1] - rows(v)[0], ranks[v]), complex)
    for a, b, ru0, rw0, su, sw, col, l in far.tolist():
        U = rng.standard_normal((su, R)) + 1j * rng.standard_normal((su, R))
        V = rng.standard_normal((sw, R)) + 1j * rng.standard_normal((sw, R))
        Fs[a][ru0:ru0 + su, col:col + R] = U
        Fs[b][rw0:rw0 + sw, col:col + R] = V
        r0, c0 = rows(a)[0] + ru0, rows(b)[0] + rw0
        T[r0:r0 + su, c0:c0 + sw] = U @ V.T
    for a, b, ca0, na, nb, col in near.tolist():
        D = rng.standard_normal((na, nb)) + 1j * rng.standard_normal((na, nb))
        Fs[a][ca0:ca0 + na, col:col + nb] = D
        Fs[b][0:nb, col:col + nb] = np.eye(nb)
        r0, c0 = rows(a)[0] + ca0, rows(b)[0]
        T[r0:r0 + na, c0:c0 + nb] = D
    T = T + T.T          # symmetric: the (b, a) blocks are the transposes
    for k in range(1 << L):
        lo, hi = ct.range(L, k)
        B = rng.standard_normal((hi - lo, hi - lo))
        T[lo:hi, lo:hi] = B + B.T
    # rebuild from the weak layout
    W = np.zeros((n, n), complex)
    for k in range(1 << L):
        lo, hi = ct.range(L, k)
        W[lo:hi, lo:hi] = T[lo:hi, lo:hi]
    for a in range(2, 1 << (L + 1), 2):
        b = a + 1
        (alo, ahi), (blo, bhi) = rows(a), rows(b)
        blk = Fs[a] @ Fs[b].T
        W[alo:ahi, blo:bhi] = blk
        W[blo:bhi, alo:ahi] = blk.T
    assert np.abs(W - T).max() <= 1e-12 * np.abs(T).max()


def test_test_vectors_are_complex_standard_normals(hs):
    # Box-Muller on Philox4x32-10: real and imaginary parts independent N(0, 1); different
    # blocks, layers and seeds give different draws; the same arguments the same draws
    scipy_stats = pytest.importorskip("scipy.stats")
    Z = np.concatenate([hs.rsvd_normals(b, 7, 0, 4096, 16).ravel() for b in range(4)])
    x = np.concatenate([Z.real, Z.imag])
    N = x.size
    assert abs(x.mean()) < 5 / np.sqrt(N)
    assert abs(x.var() - 1) < 5 * np.sqrt(2 / N)
    assert abs(np.corrcoef(Z.real, Z.imag)[0, 1]) < 5 / np.sqrt(Z.size)
    assert scipy_stats.kstest(x, "norm").pvalue > 1e-4
    a = hs.rsvd_normals(1, 2, 3, 64, 10)
    assert np.array_equal(a, hs.rsvd_normals(1, 2, 3, 64, 10))
    for other in (hs.rsvd_normals(2, 2, 3, 64, 10), hs.rsvd_normals(1, 3, 3, 64, 10), hs.rsvd_normals(1, 2, 4, 64, 10)):
        assert np.abs(a - other).min() > 0
