"""Full-size GPU checks of the workloads the bench and the method are specified at.

n = 1023 (random medium, batched point sources, mixed precision): against the oracle's
direct solve for one source and through the FP64 true residual for the batch.
n = 511 gradient (32 sources, receivers on one row): against the oracle's dense adjoint and
central differences at 16 seeded nodes, FP64 and mixed.
n = 2047 (random medium, 16 sources, mixed): the FP64 true residual, a property that holds
at any size.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import synth
from oracle.assemble import Discretization
from oracle.direct import SparseLU
from oracle import adjoint

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import paper_1007_4290_gb300 as m
    return m


def _true_relres(disc, U, F):
    A = disc.matrix()
    R = F - (A @ U.T).T
    return np.linalg.norm(R, axis=1) / np.linalg.norm(F, axis=1)


def test_n1023_random_batched_mixed(hs):
    # eight of the workload's 64 point sources in one batched mixed-precision solve, every
    # one against the direct solve of A u = f (one sparse LU of A) at the metric's relative
    # error 1e-6, and through the FP64 true residual
    w = synth.workload("n1023_random")
    n, omega, pml = w["n"], w["omega"], w["pml"]
    F = w["f"][:8].reshape(8, n * n)
    disc = Discretization(w["c"], omega, pml)
    h = hs.hsweep_setup(torch.tensor(w["c"], device="cuda"), omega, pml, w["eps_H"], hs.default_opts(precision=hs.MIXED))
    U, it, rr = h.solve(torch.tensor(F, device="cuda"), 1e-7)
    U = U.cpu().numpy()
    h.free()
    rel = _true_relres(disc, U, F)
    assert np.all(rel < 1e-6), (rel, it)
    assert max(it) <= 12
    lu = spla.splu(disc.matrix().tocsc())
    errs = []
    for s in range(8):
        u_ref = lu.solve(F[s])
        errs.append(np.linalg.norm(U[s] - u_ref) / np.linalg.norm(u_ref))
    assert max(errs) < 1e-6, errs


@pytest.fixture(scope="module")
def grad_problem():
    w = synth.workload("n511_grad")
    n, omega, pml = w["n"], w["omega"], w["pml"]
    F = w["f"].reshape(w["f"].shape[0], n * n)
    rec = w["rec_idx"]
    lu_true = SparseLU(Discretization(w["c_true"], omega, pml))
    d = np.stack([lu_true.solve(f)[rec] for f in F])
    J_ref, g_ref, _ = adjoint.misfit_and_gradient(w["c"], omega, pml, F, rec, d)
    return w, F, rec, d, J_ref, g_ref


@pytest.mark.parametrize("prec,tol", [(0, 1e-7), (1, 1e-4)])
def test_n511_gradient_against_dense_adjoint(hs, grad_problem, prec, tol):
    w, F, rec, d, J_ref, g_ref = grad_problem
    h = hs.hsweep_setup(torch.tensor(w["c"], device="cuda"), w["omega"], w["pml"], w["eps_H"],
                        hs.default_opts(precision=prec))
    J, g = h.grad(torch.tensor(F, device="cuda"), torch.tensor(rec), torch.tensor(d, device="cuda"), 1e-10)
    h.free()
    g = g.cpu().numpy().reshape(g_ref.shape)
    assert abs(J - J_ref) / J_ref < tol
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < tol


def test_n511_gradient_against_central_differences(hs, grad_problem):
    # J(c +- delta e_i) changes only A_ii; with the LU of A(c) the perturbed solves follow
    # from Sherman-Morrison: A'^{-1} f = u - alpha u_i A^{-1} e_i / (1 + alpha (A^{-1})_ii).
    w, F, rec, d, J_ref, g_ref = grad_problem
    n, omega, pml = w["n"], w["omega"], w["pml"]
    c = w["c"]
    h = hs.hsweep_setup(torch.tensor(c, device="cuda"), omega, pml, w["eps_H"], hs.default_opts(precision=hs.FP64))
    _, g = h.grad(torch.tensor(F, device="cuda"), torch.tensor(rec), torch.tensor(d, device="cuda"), 1e-10)
    h.free()
    g = g.cpu().numpy()
    disc = Discretization(c, omega, pml)
    lu = SparseLU(disc)
    U = np.stack([lu.solve(f) for f in F])
    s1s2 = disc.s1s2.ravel()
    rng = np.random.default_rng(4)
    delta = 1e-6
    interior = [j * n + i for j in range(pml + 2, n - pml - 2) for i in range(pml + 2, n - pml - 2)]
    for flat in rng.choice(interior, size=16, replace=False):
        e = np.zeros(disc.N, complex)
        e[flat] = 1.0
        col = lu.solve(e)
        Js = []
        for sgn in (1, -1):
            ci = c.ravel()[flat] + sgn * delta
            alpha = omega ** 2 / (s1s2[flat] * ci * ci) - omega ** 2 / (s1s2[flat] * c.ravel()[flat] ** 2)
            up = U - np.outer(alpha * U[:, flat] / (1 + alpha * col[flat]), col)
            r = up[:, rec] - d
            Js.append(0.5 * np.vdot(r, r).real)
        fd = (Js[0] - Js[1]) / (2 * delta)
        assert abs(fd - g[flat]) <= 1e-4 * np.max(np.abs(g)) + 1e-6 * abs(g[flat]), (flat, fd, g[flat])


def test_n2047_random_mixed_residual(hs):
    w = synth.workload("n2047_random")
    n, omega, pml = w["n"], w["omega"], w["pml"]
    F = w["f"].reshape(w["f"].shape[0], n * n)
    h = hs.hsweep_setup(torch.tensor(w["c"], device="cuda"), omega, pml, w["eps_H"], hs.default_opts(precision=hs.MIXED))
    U, it, rr = h.solve(torch.tensor(F, device="cuda"), 1e-7)
    U = U.cpu().numpy()
    h.free()
    rel = _true_relres(Discretization(w["c"], omega, pml), U, F)
    assert np.all(rel < 1e-6), (rel, it)
    np.testing.assert_allclose(rel, rr, rtol=1e-3, atol=1e-12)
