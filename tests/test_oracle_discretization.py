"""Pins for oracle O1 (assembly, Eq. sigma / Eq. helmd) and O2 (direct solve).

Each pin compares the oracle with something other than itself: exact symmetry,
the discrete sine transform solution of the un-stretched problem, a separable
fast-diagonalisation solve of the stretched constant-c problem, and second-order
convergence to a manufactured smooth solution of the continuous operator.
"""
import numpy as np
import pytest
import scipy.fft

import synth
from oracle.assemble import Discretization, pml_sigma
from oracle.direct import SparseLU, solve_banded_lu


def test_A_is_symmetric_bit_for_bit():
    # Section 2.1: after dividing by s1 s2 the operator is symmetric (A^t = A).
    n = 23
    c = synth.velocity_random(n, 1 / 8, seed=3)
    disc = Discretization(c, 2 * np.pi * 3, 5)
    A = disc.matrix()
    D = (A - A.T).tocoo()
    assert D.nnz == 0 or np.max(np.abs(D.data)) == 0.0
    assert A.nnz == 5 * n * n - 4 * n


def test_sigma_profile():
    # Eq. sigma: quadratic, C/eta at the outer boundary, zero (with zero slope) at eta.
    eta, C = 0.125, 2 * np.pi
    t = np.array([0.0, eta / 2, eta, 0.5, 1 - eta, 1 - eta / 2, 1.0])
    s = pml_sigma(t, eta, C)
    np.testing.assert_allclose(s, [C / eta, C / eta / 4, 0, 0, 0, C / eta / 4, C / eta], rtol=1e-14)
    s_lit = pml_sigma(t, eta, C, pml_form="literal")
    np.testing.assert_allclose(s_lit, s * eta, rtol=1e-14)


@pytest.mark.parametrize("n", [15, 32])
def test_unstretched_problem_matches_sine_transform(n):
    # With sigma = 0 and constant c, A = (K (x) I + I (x) K)/h^2 + omega^2/c^2 with K the
    # Dirichlet second difference; its eigenvectors are sin(k pi x), eigenvalues
    # -4 sin^2(k pi h / 2) / h^2.  Solve by DST-I and compare with both direct solvers.
    c0, omega = 1.3, 2 * np.pi * 2.7
    disc = Discretization(synth.velocity_constant(n, c0), omega, pml_width=4, C=0.0)
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(0)
    F = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    k = np.arange(1, n + 1)
    lam = -4.0 * np.sin(k * np.pi * h / 2) ** 2 / h ** 2
    denom = lam[None, :] + lam[:, None] + omega ** 2 / c0 ** 2
    Fh = scipy.fft.dstn(F, type=1, norm="ortho")
    U = scipy.fft.idstn(Fh / denom, type=1, norm="ortho")
    u1 = SparseLU(disc).solve(F.ravel())
    u2 = solve_banded_lu(disc, F.ravel())
    ref = np.linalg.norm(U)
    assert np.linalg.norm(u1 - U.ravel()) / ref < 1e-11
    assert np.linalg.norm(u2 - U.ravel()) / ref < 1e-11


def test_stretched_constant_c_separable_solve():
    # Constant c with PML: diag(s1 s2) A = K1 (x) I + I (x) K2 + omega^2/c^2 I, where the
    # 1D operators have entries s(x_i) s(x_{i +- 1/2}) / h^2.  Solve by diagonalising the
    # 1D operator (fast diagonalisation) and compare with the direct solve.
    n, omega, pml = 40, 2 * np.pi * 4, 6
    disc = Discretization(synth.velocity_constant(n), omega, pml)
    h = disc.h
    sn, sh = disc.s_node, disc.s_half
    K = np.zeros((n, n), complex)
    for i in range(n):
        K[i, i] = -(sn[i] * sh[i] + sn[i] * sh[i + 1]) / h ** 2
        if i > 0:
            K[i, i - 1] = sn[i] * sh[i] / h ** 2
        if i < n - 1:
            K[i, i + 1] = sn[i] * sh[i + 1] / h ** 2
    lam, V = np.linalg.eig(K)
    Vi = np.linalg.inv(V)
    rng = np.random.default_rng(1)
    F = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Ft = disc.s1s2 * F                       # S f, S = diag(s1 s2)
    Y = (Vi @ Ft @ Vi.T) / (lam[:, None] + lam[None, :] + omega ** 2)
    U = V @ Y @ V.T
    u = SparseLU(disc).solve(F.ravel())
    assert np.linalg.norm(u - U.ravel()) / np.linalg.norm(U) < 1e-9


def _manufactured(n, omega, pml, C):
    """f = L u* for u* = sin(pi x1) sin(pi x2) exp(x1 x2) and the continuous operator
    L u = d1((s1/s2) d1 u) + d2((s2/s1) d2 u) + omega^2 u / (s1 s2 c^2), c = 1."""
    x, h = synth.grid(n)
    eta = pml * h

    def s_and_ds(t):
        sig = pml_sigma(t, eta, C)
        dsig = np.zeros_like(t)
        if eta > 0:
            L, R = t < eta, t > 1 - eta
            dsig[L] = 2 * C / eta ** 3 * (t[L] - eta)
            dsig[R] = 2 * C / eta ** 3 * (t[R] - 1 + eta)
        s = 1.0 / (1.0 + 1j * sig / omega)
        return s, -(1j * dsig / omega) * s * s

    X1, X2 = np.meshgrid(x, x, indexing="xy")
    S1, S2, C1, C2 = np.sin(np.pi * X1), np.sin(np.pi * X2), np.cos(np.pi * X1), np.cos(np.pi * X2)
    E = np.exp(X1 * X2)
    u = S1 * S2 * E
    u1 = S2 * E * (np.pi * C1 + X2 * S1)
    u11 = S2 * E * (2 * np.pi * X2 * C1 + (X2 ** 2 - np.pi ** 2) * S1)
    u2 = S1 * E * (np.pi * C2 + X1 * S2)
    u22 = S1 * E * (2 * np.pi * X1 * C2 + (X1 ** 2 - np.pi ** 2) * S2)
    s1, ds1 = s_and_ds(X1)
    s2, ds2 = s_and_ds(X2)
    f = (ds1 * u1 + s1 * u11) / s2 + (ds2 * u2 + s2 * u22) / s1 + omega ** 2 * u / (s1 * s2)
    return u, f


@pytest.mark.parametrize("with_pml", [False, True])
def test_second_order_convergence_to_smooth_solution(with_pml):
    # Eq. helmd is a second-order scheme: the nodal error to a smooth exact solution of
    # the continuous stretched operator falls about 4x per halving of h.
    omega = 2 * np.pi * 1.5
    errs = []
    # the stretched case is in the asymptotic range from 8 cells across the PML (n = 63)
    for n in ((63, 127, 255) if with_pml else (15, 31, 63, 127)):
        pml = (n + 1) // 8 if with_pml else 0
        C = 2 * np.pi if with_pml else 0.0
        u, f = _manufactured(n, omega, pml, C)
        disc = Discretization(synth.velocity_constant(n), omega, pml, C)
        uh = SparseLU(disc).solve(f.ravel()).reshape(n, n)
        errs.append(np.max(np.abs(uh - u)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)
    assert errs[-1] < 1e-3


@pytest.mark.parametrize("n,pml", [(15, 3), (32, 5)])
def test_reflection_in_x2_maps_the_operator_onto_itself(n, pml):
    # The downward sweep (Section 3.1) factors the problem of the reflected velocity
    # c(x1, 1 - x2): its operator must be P A P, with P the reversal of the layer order,
    # and its solution the reflection of A^{-1} f.  The PML and the grid x = (k+1) h are
    # symmetric under x2 -> 1 - x2 (up to rounding of the node coordinates).
    c = synth.velocity_random(n, 1 / 8, 7)
    omega = 2 * np.pi * (n + 1) / 10
    A = Discretization(c, omega, pml).matrix().toarray()
    Ar = Discretization(c[::-1, :].copy(), omega, pml).matrix().toarray()
    perm = (np.arange(n)[::-1, None] * n + np.arange(n)[None, :]).ravel()
    PAP = A[np.ix_(perm, perm)]
    assert np.max(np.abs(Ar - PAP)) <= 1e-12 * np.max(np.abs(A))
    rng = np.random.default_rng(n)
    f = rng.standard_normal(n * n) + 1j * rng.standard_normal(n * n)
    u = SparseLU(Discretization(c, omega, pml)).solve(f)
    ur = SparseLU(Discretization(c[::-1, :].copy(), omega, pml)).solve(f[perm])
    assert np.linalg.norm(ur[perm] - u) <= 1e-10 * np.linalg.norm(u)


@pytest.mark.parametrize("k", [1, 3])
def test_dirichlet_data_on_top_matches_the_closed_form(k):
    # Section 2.5: non-zero Dirichlet data u(x1, 1) = b(x1) becomes a forcing term on the
    # last layer.  Constant c, no PML on any side, f = 0, b = sin(k pi x1): the discrete
    # solution is sin(k pi x_i) phi_j with phi_{j+1} + phi_{j-1} = 2 cos(theta) phi_j,
    # phi_0 = 0, phi_{n+1} = 1, i.e. phi_j = sin(theta j) / sin(theta (n+1)), where
    # cos(theta) = 1 - h^2 (omega^2/c^2 - lambda_k)/2 and lambda_k = (4/h^2) sin^2(k pi h/2).
    n, c0 = 31, 1.0
    h = 1.0 / (n + 1)
    omega = 2 * np.pi * 3.3
    x = (np.arange(n) + 1.0) * h
    disc = Discretization(np.full((n, n), c0), omega, 6, pml_sides=0)
    b = np.sin(k * np.pi * x)
    f = disc.boundary_rhs(3, b)
    u = SparseLU(disc).solve(f.ravel()).reshape(n, n)
    lam = 4.0 / h ** 2 * np.sin(k * np.pi * h / 2) ** 2
    theta = np.arccos(complex(1.0 - h * h * (omega ** 2 / c0 ** 2 - lam) / 2))
    j = np.arange(1, n + 1)
    phi = np.sin(theta * j) / np.sin(theta * (n + 1))
    exact = phi[:, None] * np.sin(k * np.pi * x)[None, :]
    assert np.max(np.abs(u - exact)) <= 1e-10 * np.max(np.abs(exact))


def test_pml_side_mask():
    # all four sides reproduce the default operator; no side equals no layer at all;
    # a layer on x1 = 0 only is the mirror image (x1 -> 1 - x1) of a layer on x1 = 1 only
    n, pml = 24, 5
    c = synth.velocity_random(n, 1 / 6, 11)
    omega = 2 * np.pi * 4.1
    A = Discretization(c, omega, pml).matrix()
    assert (Discretization(c, omega, pml, pml_sides=15).matrix() != A).nnz == 0
    assert (Discretization(c, omega, pml, pml_sides=0).matrix() != Discretization(c, omega, 0).matrix()).nnz == 0
    A_left = Discretization(c, omega, pml, pml_sides=1).matrix().toarray()
    A_right = Discretization(c[:, ::-1].copy(), omega, pml, pml_sides=2).matrix().toarray()
    perm = (np.arange(n)[:, None] * n + np.arange(n)[::-1][None, :]).ravel()
    assert np.max(np.abs(A_left - A_right[np.ix_(perm, perm)])) <= 1e-12 * np.max(np.abs(A_left))
    for sides in (1, 6, 9):
        M = Discretization(c, omega, pml, pml_sides=sides).matrix()
        assert abs(M - M.T).max() == 0
