"""Pins for the strongly admissible H-matrices of the oracle (Section 2.3, the strongly
admissible case) and the H-sweep built on them (Algorithms 2.5/2.6).

Pinned against: the paper's geometric definition of well-separatedness evaluated on the
index ranges, brute-force coverage of the block partition, dense products and inverses
(numpy), the exact sweep (dense Algorithm 2.1), the rank-r recovery property and the
expected-error bound of the randomized SVD (Halko, Martinsson and Tropp, Theorem 10.5),
and the direct solve.
"""
import numpy as np
import pytest

import synth
from oracle import hmatrix_strong as hs
from oracle.assemble import Discretization
from oracle.direct import SparseLU
from oracle.gmres import preconditioned_solve
from oracle.hmatrix import Trunc
from oracle.sweep_exact import setup_exact, solve_exact
from oracle.sweep_h import HSweep


def _rand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("n,leaf", [(64, 4), (63, 4), (127, 8), (37, 5)])
def test_well_separated_blocks_follow_the_geometric_definition(n, leaf):
    # Section 2.3: two clusters are well separated when the distance between them is at
    # least their width.  Grid points x_k = (k + 1) h; a cluster [lo, hi) spans
    # (hi - 1 - lo) h, and the distance between [lo, hi) and [lo', hi') (hi <= lo') is
    # (lo' - hi + 1) h.  Every factorised block must satisfy it for both clusters, every
    # refined or dense block must violate it, and the blocks must tile the matrix.  (The
    # index rule |i - i'| >= 2 and the geometric one agree while clusters hold at least
    # three indices, as with every leaf size used here.)
    ct = hs.Clusters(n, leaf)
    G = _rand(np.random.default_rng(0), n, n)
    root = hs.from_dense(ct, G, Trunc())
    cover = np.zeros((n, n), int)

    def visit(B):
        rlo, rhi = ct.range(B.l, B.i)
        clo, chi = ct.range(B.l, B.j)
        if rhi <= clo:
            dist = clo - rhi + 1
        elif chi <= rlo:
            dist = rlo - chi + 1
        else:
            dist = 0
        sep = dist >= (rhi - 1 - rlo) and dist >= (chi - 1 - clo)
        if B.kind == "F":
            assert sep
            cover[rlo:rhi, clo:chi] += 1
        elif B.kind == "D":
            assert not sep and B.l == ct.L
            cover[rlo:rhi, clo:chi] += 1
        else:
            assert not sep and B.l < ct.L
            for a in (0, 1):
                for b in (0, 1):
                    visit(B.ch[a][b])

    visit(root)
    assert (cover == 1).all()
    assert np.abs(root.to_dense() - G).max() < 1e-12 * np.abs(G).max()


def test_interaction_lists_are_symmetric_and_at_most_three():
    # the interaction list is a symmetric relation (Section 2.3); in one dimension it has
    # at most three members, and the factorised blocks of an H-matrix are exactly the
    # (i, j) with j in the interaction list of i
    ct = hs.Clusters(128, 4)
    G = _rand(np.random.default_rng(1), 128, 128)
    root = hs.from_dense(ct, G, Trunc())
    blocks = {(l, i, j) for l, i, j, _, _ in root.factor_blocks()}
    listed = set()
    for l in range(ct.L + 1):
        for i in range(1 << l):
            il = ct.interaction_list(l, i)
            assert len(il) <= 3
            for j in il:
                assert i in ct.interaction_list(l, j)
                listed.add((l, i, j))
    assert blocks == listed
    # the interior clusters of depth >= 2 have exactly three
    assert all(len(ct.interaction_list(4, i)) == 3 for i in range(2, 14))


@pytest.mark.parametrize("n,leaf", [(64, 4), (45, 4)])
def test_strong_h_operations_are_exact_without_truncation(n, leaf):
    # eps = 0, no rank cap: hmatvec, hadd, hmul (all eight forms, F = H.H by the
    # randomized SVD with a full set of test vectors), hdiagmul and hinv reproduce the
    # dense operations.
    rng = np.random.default_rng(n)
    ct = hs.Clusters(n, leaf)
    tr = Trunc()
    G, H = _rand(rng, n, n), _rand(rng, n, n)
    Gh, Hh = hs.from_dense(ct, G, tr), hs.from_dense(ct, H, tr)
    x = _rand(rng, n, 3)
    assert np.abs(Gh.matvec(x) - G @ x).max() < 1e-12 * np.abs(G @ x).max()
    assert np.abs(Gh.rmatvec(x) - G.T @ x).max() < 1e-12 * np.abs(G.T @ x).max()
    assert np.abs(hs.hadd(Gh, Hh, tr, 0.5).to_dense() - (G + 0.5 * H)).max() < 1e-12 * np.abs(G).max()
    P = G @ H
    assert np.abs(hs.hmul(Gh, Hh, tr, rng).to_dense() - P).max() < 1e-11 * np.abs(P).max()
    d1, d2 = _rand(rng, n), _rand(rng, n)
    assert np.abs(Gh.diagmul(d1, d2).to_dense() - d1[:, None] * G * d2[None, :]).max() < 1e-12 * np.abs(G).max() * 10
    A = G + 3 * np.sqrt(n) * np.eye(n)
    Ainv = np.linalg.inv(A)
    X = hs.hinv(hs.from_dense(ct, A, tr), tr, rng).to_dense()
    assert np.abs(X - Ainv).max() < 1e-11 * np.abs(Ainv).max()


def test_hmul_exercises_the_randomized_product():
    # F = H . H occurs: a well-separated position whose operands are both hierarchical
    # (depth 2: (0, 1) times (1, 2) lands on (0, 2)); it must be exact for a product of
    # rank r with r test vectors plus oversampling.
    rng = np.random.default_rng(7)
    ct = hs.Clusters(64, 4)
    tr = Trunc()
    G, H = _rand(rng, 64, 64), _rand(rng, 64, 64)
    Gb = hs.from_dense(ct, G[0:16, 16:32], tr, 2, 0, 1)
    Hb = hs.from_dense(ct, H[16:32, 32:48], tr, 2, 1, 2)
    assert Gb.kind == "H" and Hb.kind == "H" and ct.kind(2, 0, 2) == "F"
    R = hs.hmul(Gb, Hb, tr, rng)
    assert R.kind == "F"
    ref = G[0:16, 16:32] @ H[16:32, 32:48]
    assert np.abs(R.to_dense() - ref).max() < 1e-12 * np.abs(ref).max()


def test_randomized_svd_recovers_rank_r_exactly_and_meets_the_error_bound():
    # (1) a product of exact rank r is recovered to rounding with rmax = r;
    # (2) for a product with singular values s_j = 2^-j, the rank-r approximation error
    #     stays within the expected-error bound of Halko, Martinsson and Tropp
    #     (Theorem 10.5 with p oversampling columns): E||A - QQ*A|| <= (1 + sqrt(r/(p-1)))
    #     s_{r+1} + e sqrt(r+p)/p (sum_{j>r} s_j^2)^{1/2}; we ask for 3x that bound, and the
    #     truncation to rank r adds at most s_{r+1} more.
    rng = np.random.default_rng(11)
    ct = hs.Clusters(64, 4)
    m = 16
    X, Y = _rand(rng, m, 3), _rand(rng, m, 3)
    W = np.linalg.qr(_rand(rng, m, m))[0]
    G = hs.from_dense(ct, X @ Y.T, Trunc(), 2, 0, 1)
    H = hs.from_dense(ct, W, Trunc(), 2, 1, 2)
    U, V = hs.rsvd_product(G, H, Trunc(0.0, 3), rng)
    ref = X @ Y.T @ W
    assert np.abs(U @ V.T - ref).max() < 1e-12 * np.abs(ref).max()

    s = 2.0 ** -np.arange(m)
    Q1, Q2 = np.linalg.qr(_rand(rng, m, m))[0], np.linalg.qr(_rand(rng, m, m))[0]
    A = (Q1 * s) @ Q2.T
    G = hs.from_dense(ct, A, Trunc(), 2, 0, 1)
    H = hs.from_dense(ct, np.eye(m, dtype=complex), Trunc(), 2, 1, 2)
    r, p = 2, hs.RSVD_OVERSAMPLE
    bound = (1 + np.sqrt(r / (p - 1))) * s[r] + np.e * np.sqrt(r + p) / p * np.sqrt(np.sum(s[r:] ** 2))
    errs = []
    for _ in range(20):
        U, V = hs.rsvd_product(G, H, Trunc(0.0, r), rng)
        assert U.shape[1] == r
        errs.append(np.linalg.norm(A - U @ V.T, 2))
    assert np.mean(errs) <= 3 * bound + s[r]
    assert min(errs) >= s[r] * (1 - 1e-9)           # no rank-r matrix does better (Eckart-Young)


def test_tridiagonal_block_is_exact_with_rank_zero_far_field():
    ct = hs.Clusters(37, 4)
    rng = np.random.default_rng(2)
    d, e = _rand(rng, 37), _rand(rng, 36)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    B = hs.tridiag(ct, d, e)
    assert np.abs(B.to_dense() - T).max() == 0.0
    assert all(U.shape[1] == 0 for _, _, _, U, _ in B.factor_blocks())


def test_strong_h_sweep_without_truncation_is_the_exact_sweep():
    n = 31
    disc = Discretization(synth.velocity_random(n, 1 / 8, 0), 2 * np.pi * 32 / 12.0, 4)
    T = setup_exact(disc)
    f = _rand(np.random.default_rng(3), disc.N)
    ref = solve_exact(disc, T, f)
    S = HSweep(disc, 0.0, leaf=4, admissibility="strong")
    u = S.apply(f)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-11


def test_strong_rank_two_preconditioner_converges_where_weak_rank_two_is_slower():
    # Section 3 uses the strongly admissible case with R = 2: on the mixed-boundary
    # example (Dirichlet at x1 = 0 and 1) the strong preconditioner reaches 1e-3 in a few
    # steps, fewer than the weak one at the same rank, and GMRES reaches the direct
    # solution at a tight tolerance.
    w = synth.workload("mixed1_n63")
    disc = Discretization(w["c"], w["omega"], w["pml"], pml_sides=w["pml_sides"])
    A = disc.matrix()
    f = w["f"].reshape(-1)
    its = {}
    for adm in ("weak", "strong"):
        S = HSweep(disc, 0.0, leaf=8, rmax=2, admissibility=adm)
        _, its[adm], _ = preconditioned_solve(A, S.apply, f, 1e-3, 100)
    assert its["strong"] <= 3 and its["strong"] < its["weak"]
    S = HSweep(disc, 0.0, leaf=8, rmax=2, admissibility="strong")
    u, _, _ = preconditioned_solve(A, S.apply, f, 1e-12, 100)
    u_ref = SparseLU(disc).solve(f)
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-9


def _paper_steps():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_gmres_steps.txt")
    out = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            key, om, q, n1, t1, t2 = line.split()
            out[(key, int(n1), int(q))] = (int(t1), int(t2))
    return out


@pytest.mark.parametrize("field", [1, 2, 3])
def test_strong_rank_two_sweep_takes_the_papers_steps_at_n_plus_1_128(field):
    # the tables of Section 3.1 (dependence on omega) at omega / 2 pi = 16, q = 8: the
    # oracle's strongly admissible H-sweep with R = 2 on the synthetic stand-ins for the
    # pictured fields (synth.workload('pml{field}_n127')) takes the printed GMRES steps
    # for both forces at tolerance 1e-3
    want = _paper_steps()[("pml_field%d" % field, 128, 8)]
    w = synth.workload("pml%d_n127" % field)
    disc = Discretization(w["c"], w["omega"], w["pml"])
    A = disc.matrix()
    S = HSweep(disc, 0.0, leaf=8, rmax=2, admissibility="strong")
    got = tuple(preconditioned_solve(A, S.apply, w["f"][s].ravel(), 1e-3, 50)[1] for s in range(2))
    assert got == want, (got, want)


def test_rank_R_form_of_a_dense_matrix_is_the_blockwise_truncated_svd():
    # from_dense with a rank cap R keeps, on every block of an interaction list, the best
    # rank-R approximation (Eckart-Young: the error is the (R+1)-th singular value), and
    # every dense block exactly
    rng = np.random.default_rng(21)
    n, R = 64, 2
    ct = hs.Clusters(n, 4)
    x = np.arange(n) / n
    G = 1.0 / (1.0 + 40 * np.abs(x[:, None] - x[None, :])) + 0.01 * _rand(rng, n, n)
    B = hs.from_dense(ct, G, Trunc(0.0, R))
    for l, i, j, U, V in B.factor_blocks():
        r0, r1 = ct.range(l, i)
        c0, c1 = ct.range(l, j)
        blk = G[r0:r1, c0:c1]
        s = np.linalg.svd(blk, compute_uv=False)
        assert U.shape[1] <= R
        assert abs(np.linalg.norm(blk - U @ V.T, 2) - s[R]) <= 1e-10 * s[0]
    for l, i, j, D in B.dense_blocks():
        r0, r1 = ct.range(l, i)
        c0, c1 = ct.range(l, j)
        assert np.array_equal(D, G[r0:r1, c0:c1])
