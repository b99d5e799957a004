"""GPU parity of the adjoint gradient of the misfit 1/2 sum_s ||R u_s - d_s||^2 with
respect to c: against the oracle's dense adjoint (sparse LU, conjugate-transposed
solve), against central finite differences of the oracle misfit, and through the
torch.autograd wrapper."""
import numpy as np
import pytest
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


def _problem(n=63, nsrc=4):
    omega, pml = 2 * np.pi * 5, 8
    c_true = synth.velocity_lens(n)
    c = c_true + 0.05 * synth.smooth_noise(n, 1 / 16, 3)
    _, h = synth.grid(n)
    xs = pml * h + (np.arange(nsrc) + 0.5) * (1 - 2 * pml * h) / nsrc
    F = np.stack([synth.source_delta(n, (x, 0.8)).ravel() for x in xs])
    rec = (int(0.7 * (n + 1)) - 1) * n + np.arange(n)
    lu = SparseLU(Discretization(c_true, omega, pml))
    d = np.stack([lu.solve(f)[rec] for f in F])
    return c, omega, pml, F, rec, d


@pytest.mark.parametrize("prec,tol", [(0, 1e-8), (1, 1e-4)])
def test_gradient_matches_oracle_dense_adjoint(hs, prec, tol):
    c, omega, pml, F, rec, d = _problem()
    J_ref, g_ref, _ = adjoint.misfit_and_gradient(c, omega, pml, F, rec, d)
    h = hs.hsweep_setup(torch.tensor(c, device="cuda"), omega, pml, 1e-8, hs.default_opts(precision=prec))
    J, g = h.grad(torch.tensor(F, device="cuda"), torch.tensor(rec), torch.tensor(d, device="cuda"), 1e-11)
    h.free()
    g = g.cpu().numpy().reshape(c.shape)
    assert abs(J - J_ref) / J_ref < tol
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < tol


def test_gradient_matches_central_differences(hs):
    c, omega, pml, F, rec, d = _problem()
    h = hs.hsweep_setup(torch.tensor(c, device="cuda"), omega, pml, 1e-8, hs.default_opts(precision=0))
    _, g = h.grad(torch.tensor(F, device="cuda"), torch.tensor(rec), torch.tensor(d, device="cuda"), 1e-11)
    h.free()
    g = g.cpu().numpy().reshape(c.shape)
    n = c.shape[0]
    rng = np.random.default_rng(4)
    delta = 1e-6
    for flat in rng.choice(np.arange(10 * n, n * n - 10 * n), size=8, replace=False):
        j, i = divmod(int(flat), n)
        cp, cm = c.copy(), c.copy()
        cp[j, i] += delta
        cm[j, i] -= delta
        fd = (adjoint.misfit(cp, omega, pml, F, rec, d) - adjoint.misfit(cm, omega, pml, F, rec, d)) / (2 * delta)
        assert abs(fd - g[j, i]) <= 1e-5 * np.max(np.abs(g)), (j, i, fd, g[j, i])


def test_autograd_function(hs):
    from paper_1007_4290_gb300.autograd import helmholtz_misfit
    c, omega, pml, F, rec, d = _problem(n=31, nsrc=2)
    ct = torch.tensor(c, device="cuda", requires_grad=True)
    J = helmholtz_misfit(ct, torch.tensor(F, device="cuda"), torch.tensor(rec), torch.tensor(d, device="cuda"),
                         omega, pml, 1e-8, 1e-11, hs.default_opts(precision=0))
    (2.0 * J).backward()
    J_ref, g_ref, _ = adjoint.misfit_and_gradient(c, omega, pml, F, rec, d)
    assert abs(J.item() - J_ref) / J_ref < 1e-8
    g = ct.grad.cpu().numpy()
    assert np.linalg.norm(g - 2 * g_ref) / np.linalg.norm(2 * g_ref) < 1e-8
