"""Pins for oracle O3 (exact sweep, Algorithms 2.1/2.2), O4 (H-algebra and the
H-sweep, Section 2.3, Algorithms 2.5/2.6), GMRES and the adjoint gradient.

Pinned against: dense inversion (numpy), the half-space Green's function identity
(Eq. Afacminv), brute-force SVDs of every block, dense products, finite
differences of the misfit, and a Taylor remainder test.
"""
import numpy as np
import pytest

import synth
from oracle.assemble import Discretization
from oracle.direct import SparseLU
from oracle.sweep_exact import setup_exact, solve_exact
from oracle.hmatrix import (HMatrix, Trunc, tree_depth, hadd, hsub, hmul, hinv,
                            add_lowrank, recompress)
from oracle.sweep_h import HSweep
from oracle.gmres import gmres, preconditioned_solve
from oracle import adjoint


def _disc(n, seed=0, pml=None, C=2 * np.pi, ppw=12.0):
    c = synth.velocity_random(n, 1 / 8, seed) if seed is not None else synth.velocity_constant(n)
    omega = 2 * np.pi * (n + 1) / ppw
    return Discretization(c, omega, pml if pml is not None else max(2, (n + 1) // 8), C)


def test_tree_depths_of_the_workloads():
    assert [tree_depth(n, 8) for n in (64, 511, 1023, 2047, 8, 9, 17)] == [3, 6, 7, 8, 0, 1, 2]


# --- O3 ----------------------------------------------------------------------------
@pytest.mark.parametrize("n", [7, 16, 31])
def test_exact_sweep_reproduces_dense_inverse(n):
    # Eq. Afact: the block LDL^t sweep is an exact factorisation of A.
    disc = _disc(n)
    T = setup_exact(disc)
    Ainv = np.linalg.inv(disc.matrix().toarray())
    rng = np.random.default_rng(n)
    f = rng.standard_normal(disc.N) + 1j * rng.standard_normal(disc.N)
    u = solve_exact(disc, T, f)
    assert np.linalg.norm(u - Ainv @ f) / np.linalg.norm(Ainv @ f) < 1e-12
    # column by column: the sweep applied to the identity is A^{-1}
    E = np.eye(disc.N)[:, :: max(1, disc.N // 17)]
    U = np.stack([solve_exact(disc, T, e) for e in E.T], axis=1)
    assert np.linalg.norm(U - Ainv @ E) / np.linalg.norm(Ainv @ E) < 1e-12


def test_T_m_is_the_half_space_green_function():
    # Eq. Afacminv: T_m equals the (m, m) block of the inverse of the leading m x m
    # block submatrix (the half-space problem with zero data on row m + 1).
    n = 15
    disc = _disc(n)
    T = setup_exact(disc)
    A = disc.matrix().toarray()
    for m in (1, 5, 11, 15):
        Gm = np.linalg.inv(A[: m * n, : m * n])[-n:, -n:]
        assert np.linalg.norm(T[m - 1] - Gm) / np.linalg.norm(Gm) < 1e-12


def test_sparse_and_exact_sweep_agree_at_moderate_n():
    n = 63
    disc = _disc(n, seed=2)
    f = synth.source_gaussian(n, (0.4, 0.6), 1 / 20).ravel()
    u_lu = SparseLU(disc).solve(f)
    u_sw = solve_exact(disc, setup_exact(disc), f)
    assert np.linalg.norm(u_lu - u_sw) / np.linalg.norm(u_lu) < 1e-10


# --- O4 H-algebra --------------------------------------------------------------------
def _green_like(n, seed):
    """A dense T_m from the exact sweep (the kind of matrix the method compresses),
    plus a non-symmetric perturbation so transposition mistakes show."""
    disc = _disc(n, seed=seed)
    T = setup_exact(disc)[n // 2]
    rng = np.random.default_rng(seed)
    return T + 1e-3 * np.linalg.norm(T) / n * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))


@pytest.mark.parametrize("n", [9, 24, 37])
def test_h_operations_are_exact_without_truncation(n):
    # Section 2.3: with no truncation every operation equals the dense one.
    tr = Trunc(0.0)
    G = _green_like(n, 1)
    H = _green_like(n, 2)
    hG, hH = HMatrix.from_dense(G, tr), HMatrix.from_dense(H, tr)
    ref = np.linalg.norm(G)
    assert np.linalg.norm(hG.to_dense() - G) / ref < 1e-13
    rng = np.random.default_rng(5)
    x = rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))
    np.testing.assert_allclose(hG.matvec(x), G @ x, rtol=0, atol=1e-12 * np.linalg.norm(G @ x))
    np.testing.assert_allclose(hG.rmatvec(x), G.T @ x, rtol=0, atol=1e-12 * np.linalg.norm(G.T @ x))
    assert np.linalg.norm(hadd(hG, hH, tr).to_dense() - (G + H)) / ref < 1e-12
    assert np.linalg.norm(hsub(hG, hH, tr).to_dense() - (G - H)) / ref < 1e-12
    P = G @ H
    assert np.linalg.norm(hmul(hG, hH, tr).to_dense() - P) / np.linalg.norm(P) < 1e-11
    Gi = np.linalg.inv(G)
    assert np.linalg.norm(hinv(hG, tr).to_dense() - Gi) / np.linalg.norm(Gi) < 1e-10
    dl = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    dr = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    D = hG.diagmul(dl=dl, dr=dr).to_dense()
    assert np.linalg.norm(D - dl[:, None] * G * dr[None, :]) / ref < 1e-13
    X = rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2))
    Y = rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2))
    GXY = G + X @ Y.T
    assert np.linalg.norm(add_lowrank(hG, X, Y, tr).to_dense() - GXY) / np.linalg.norm(GXY) < 1e-12


def _check_blocks_within_eps(hM, M, eps):
    for _, (r0, r1), (c0, c1), U, V in hM.blocks():
        B = M[r0:r1, c0:c1]
        s = np.linalg.svd(B, compute_uv=False)
        err = np.linalg.norm(B - U @ V.T, 2)
        assert err <= eps * s[0] * (1 + 1e-8) + 1e-14 * s[0], (r0, c0, err / s[0])
        # and no more terms than the brute-force count above the threshold
        assert U.shape[1] == int(np.count_nonzero(s > eps * s[0]))


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_truncation_error_of_every_block_is_within_eps(eps):
    # Section 2.3 recompression: a truncated block is within eps * sigma_1 in the
    # spectral norm of the block it represents (brute-force SVD of the dense block).
    n = 64
    G = setup_exact(_disc(n, seed=4))[40]
    hG = HMatrix.from_dense(G, Trunc(eps))
    _check_blocks_within_eps(hG, G, eps)
    # recompression of a sum of two exact factorisations
    H = setup_exact(_disc(n, seed=5))[40]
    hH0, hG0 = HMatrix.from_dense(H, Trunc(0.0)), HMatrix.from_dense(G, Trunc(0.0))
    S = hadd(hG0, hH0, Trunc(eps))
    _check_blocks_within_eps(S, G + H, eps)


def test_recompress_handles_rank_deficient_and_empty_input():
    rng = np.random.default_rng(0)
    U = rng.standard_normal((20, 2)) + 1j * rng.standard_normal((20, 2))
    V = rng.standard_normal((17, 2))
    Ud, Vd = recompress(np.hstack([U, U]), np.hstack([V, V]), Trunc(1e-12))
    assert Ud.shape[1] == 2
    np.testing.assert_allclose(Ud @ Vd.T, 2 * U @ V.T, atol=1e-12)
    Z = recompress(np.zeros((5, 3), complex), np.zeros((4, 3), complex), Trunc(1e-6))
    assert Z[0].shape == (5, 0) and Z[1].shape == (4, 0)


# --- O4 sweep -----------------------------------------------------------------------
def test_h_sweep_without_truncation_is_the_exact_sweep():
    n = 31
    disc = _disc(n, seed=6)
    T = setup_exact(disc)
    hs = HSweep(disc, 0.0)
    for m in (0, 9, 30):
        assert np.linalg.norm(hs.T[m].to_dense() - T[m]) / np.linalg.norm(T[m]) < 1e-10
    f = synth.source_gaussian(n, (0.5, 0.5), 1 / 16).ravel()
    u = SparseLU(disc).solve(f)
    assert np.linalg.norm(hs.apply(f) - u) / np.linalg.norm(u) < 1e-10


def test_h_sweep_error_decreases_with_eps():
    n = 63
    disc = _disc(n, seed=7)
    f = synth.source_gaussian(n).ravel()
    u = SparseLU(disc).solve(f)
    errs = [np.linalg.norm(HSweep(disc, e).apply(f) - u) / np.linalg.norm(u) for e in (1e-3, 1e-6, 1e-9)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-6


def test_ranks_smaller_with_pml_than_with_dirichlet():
    # Section 2.2 (rank maps, n = 256, omega/2pi = 32, threshold 1e-6): an absorbing
    # layer keeps the off-diagonal ranks of T_m low, zero Dirichlet data makes them
    # larger.  The contrast needs a strongly absorbing layer (here C = 40 over 32
    # cells); with C = 2 pi the layer reflects a few percent and the ranks approach
    # the Dirichlet ones.
    n = 255
    omega = 2 * np.pi * 32.3
    c = synth.velocity_constant(n)

    def ranks(C):
        T = setup_exact(Discretization(c, omega, 32, C))[n // 2]
        out = []
        for q in (128, 64):
            s = np.linalg.svd(T[:q, q:2 * q], compute_uv=False)
            out.append(int(np.count_nonzero(s > 1e-6 * s[0])))
        return out

    r_pml, r_dir = ranks(40.0), ranks(0.0)
    assert r_pml[0] < 0.7 * r_dir[0] and r_pml[1] < 0.7 * r_dir[1], (r_pml, r_dir)


# --- GMRES --------------------------------------------------------------------------
def test_gmres_solves_a_dense_system():
    rng = np.random.default_rng(3)
    n = 40
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, it, hist = gmres(lambda v: A @ v, b, 1e-12, max_it=n)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) / np.linalg.norm(x) < 1e-10
    assert it <= n and hist[-1] <= 1e-12
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1))


def test_preconditioned_gmres_matches_direct_solve():
    n = 63
    disc = _disc(n, seed=8)
    hs = HSweep(disc, 1e-4)
    f = synth.source_gaussian(n, (0.45, 0.55), 1 / 32).ravel()
    u_ref = SparseLU(disc).solve(f)
    u, it, _ = preconditioned_solve(disc.matrix(), hs.apply, f, 1e-10)
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-8
    assert it <= 6


# --- adjoint gradient ---------------------------------------------------------------
def _grad_problem(n=23):
    omega, pml = 2 * np.pi * 2.5, 4
    c_true = synth.velocity_lens(n)
    c = c_true + 0.05 * synth.smooth_noise(n, 1 / 8, 3)
    xs = [0.3, 0.5, 0.7]
    F = np.stack([synth.source_delta(n, (x, 0.8)).ravel() for x in xs])
    rec = (n * 3 // 4) * n + np.arange(n)
    lu = SparseLU(Discretization(c_true, omega, pml))
    d = np.stack([lu.solve(f)[rec] for f in F])
    return c, omega, pml, F, rec, d


def test_adjoint_gradient_matches_central_differences():
    c, omega, pml, F, rec, d = _grad_problem()
    J, g, _ = adjoint.misfit_and_gradient(c, omega, pml, F, rec, d)
    rng = np.random.default_rng(4)
    n = c.shape[0]
    delta = 1e-6
    for flat in rng.choice(n * n, size=6, replace=False):
        j, i = divmod(int(flat), n)
        cp, cm = c.copy(), c.copy()
        cp[j, i] += delta
        cm[j, i] -= delta
        fd = (adjoint.misfit(cp, omega, pml, F, rec, d) - adjoint.misfit(cm, omega, pml, F, rec, d)) / (2 * delta)
        assert abs(fd - g[j, i]) <= 1e-5 * np.max(np.abs(g)), (j, i, fd, g[j, i])


def test_adjoint_gradient_taylor_remainder_is_second_order():
    c, omega, pml, F, rec, d = _grad_problem()
    J, g, _ = adjoint.misfit_and_gradient(c, omega, pml, F, rec, d)
    dc = synth.smooth_noise(c.shape[0], 1 / 6, 9)
    rem = []
    for t in (1e-2, 5e-3, 2.5e-3):
        rem.append(abs(adjoint.misfit(c + t * dc, omega, pml, F, rec, d) - J - t * np.sum(g * dc)))
    rates = np.log2(np.array(rem[:-1]) / np.array(rem[1:]))
    assert np.all(rates > 1.8), rates
