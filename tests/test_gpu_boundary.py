"""GPU parity of the other boundary conditions (Section 2.5; the examples of Section 3.2):
a PML on some sides only (`pml_sides`), zero Dirichlet on the others, and non-zero
Dirichlet data moved into the forcing term (`hsweep_boundary_rhs`), against the oracle's
matrix, forcing term and direct solve."""
import numpy as np
import pytest
import torch

import synth
from oracle.assemble import Discretization
from oracle.direct import SparseLU

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import paper_1007_4290_gb300 as m
    return m


def _handle(hs, w, direction=1, setup=True):
    opts = hs.default_opts(precision=0, r_max=8, pml_sides=w["pml_sides"], sweep_dir=direction)
    make = hs.hsweep_setup if setup else hs.hsweep_create
    return make(torch.tensor(w["c"], device="cuda"), w["omega"], w["pml"], 1e-8, opts)


@pytest.mark.parametrize("name", ["depth1_n127", "mixed1_n127", "mixed2_n127"])
@pytest.mark.parametrize("direction", [1, -1])
def test_masked_pml_matvec_matches_oracle_matrix(hs, name, direction):
    w = synth.workload(name)
    n = w["n"]
    A = Discretization(w["c"], w["omega"], w["pml"], pml_sides=w["pml_sides"]).matrix()
    h = _handle(hs, w, direction, setup=False)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((2, n * n)) + 1j * rng.standard_normal((2, n * n))
    Y = h.matvec(torch.tensor(X, device="cuda")).cpu().numpy()
    h.free()
    ref = (A @ X.T).T
    assert np.linalg.norm(Y - ref) / np.linalg.norm(ref) < 1e-14


@pytest.mark.parametrize("direction", [1, -1])
@pytest.mark.parametrize("side", [0, 1, 2, 3])
def test_boundary_data_forcing_term_matches_oracle(hs, side, direction):
    w = synth.workload("depth2_n127")
    n = w["n"]
    disc = Discretization(w["c"], w["omega"], w["pml"], pml_sides=w["pml_sides"])
    rng = np.random.default_rng(side)
    b = rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))
    F = rng.standard_normal((2, n * n)) + 1j * rng.standard_normal((2, n * n))
    h = _handle(hs, w, direction, setup=False)
    Fg = torch.tensor(F, device="cuda")
    h.boundary_rhs(side, torch.tensor(b, device="cuda"), Fg)
    got = Fg.cpu().numpy()
    h.free()
    ref = F + np.stack([disc.boundary_rhs(side, b[s]).ravel() for s in range(2)])
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))


@pytest.mark.parametrize("name", ["depth1_n127", "depth2_n127", "mixed1_n127", "mixed2_n127"])
@pytest.mark.parametrize("direction", [1, -1])
def test_boundary_problems_solve_to_the_direct_solution(hs, name, direction):
    # both sweep directions; the downward sweeps of depth1, depth2 and mixed2 start at a
    # Dirichlet side (no absorption in the first Schur complements)
    w = synth.workload(name)
    n = w["n"]
    disc = Discretization(w["c"], w["omega"], w["pml"], pml_sides=w["pml_sides"])
    f = w["f"].reshape(1, n * n).copy()
    if "b_top" in w:
        f += disc.boundary_rhs(3, w["b_top"][0]).ravel()[None, :]
    u_ref = SparseLU(disc).solve(f[0])
    h = _handle(hs, w, direction)
    fg = torch.tensor(w["f"].reshape(1, n * n), device="cuda")
    if "b_top" in w:
        h.boundary_rhs(3, torch.tensor(w["b_top"], device="cuda"), fg)
    u, it, rr = h.solve(fg, 1e-10)
    h.free()
    u = u.cpu().numpy()[0]
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-7, it
