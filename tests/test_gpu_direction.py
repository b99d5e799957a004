"""GPU parity of the downward sweep (sweep_dir = -1; Section 3.1, the dependence on the
sweeping direction), on the workload of that test: c = 1/2 + x2, a narrow Gaussian point
source at (0.125, 0.5), q = 8 points per wavelength and fixed rank R = 2.

The downward handle factors the reflected problem; its apply is checked against the
oracle's exact sweep (Algorithm 2.2) run on the dense layers it exported, its solve against
the direct solve of the original A, and its gradient against the upward handle's."""
import numpy as np
import pytest
import torch

import synth
from oracle.assemble import Discretization
from oracle.direct import SparseLU
from oracle.sweep_exact import solve_exact
from tests.helpers import layer_to_dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import paper_1007_4290_gb300 as m
    return m


def _perm(n):
    return (np.arange(n)[::-1, None] * n + np.arange(n)[None, :]).ravel()


def _handle(hs, w, direction, prec=0, r_max=None, eps=None):
    opts = hs.default_opts(precision=prec, r_max=r_max if r_max is not None else w["r_max"], sweep_dir=direction)
    return hs.hsweep_setup(torch.tensor(w["c"], device="cuda"), w["omega"], w["pml"],
                           w["eps_H"] if eps is None else eps, opts)


@pytest.mark.parametrize("prec", [0, 1])
def test_downward_apply_matches_exact_sweep_of_the_reflected_layers(hs, prec):
    w = synth.workload("dir_n127")
    n = w["n"]
    P = _perm(n)
    h = _handle(hs, w, -1, prec=prec, r_max=8, eps=1e-8)
    rng = np.random.default_rng(3)
    R = rng.standard_normal((3, n * n)) + 1j * rng.standard_normal((3, n * n))
    Z = h.apply(torch.tensor(R, device="cuda")).cpu().numpy()
    assert h.status()[0] == 0
    T = []
    for m in range(n):
        lv, fac, rk = h.export_layer(m)
        T.append(layer_to_dense(n, 8, 8, lv, fac, rk))
    h.free()
    disc_r = Discretization(w["c"][::-1, :].copy(), w["omega"], w["pml"])
    tol = 1e-12 if prec == 0 else 2e-5
    for s in range(3):
        ref = solve_exact(disc_r, T, R[s][P])[P]
        assert np.linalg.norm(Z[s] - ref) / np.linalg.norm(ref) < tol


@pytest.mark.parametrize("direction", [1, -1])
def test_both_directions_solve_the_original_problem(hs, direction):
    w = synth.workload("dir_n127")
    n = w["n"]
    disc = Discretization(w["c"], w["omega"], w["pml"])
    f = w["f"].reshape(1, n * n)
    u_ref = SparseLU(disc).solve(f[0])
    h = _handle(hs, w, direction, r_max=8, eps=1e-8)
    u, it, rr = h.solve(torch.tensor(f, device="cuda"), 1e-10)
    u = u.cpu().numpy()[0]
    h.free()
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-7, it
    assert rr[0] < 1e-8


def test_downward_gradient_equals_upward_gradient(hs):
    w = synth.workload("dir_n127")
    n = w["n"]
    rng = np.random.default_rng(5)
    F = np.stack([synth.source_gaussian(n, (0.125 + 0.25 * k, 0.5)).ravel() for k in range(3)])
    rec = (n - 20) * n + np.arange(10, n - 10)
    d = rng.standard_normal((3, rec.size)) + 1j * rng.standard_normal((3, rec.size))
    out = {}
    for direction in (1, -1):
        h = _handle(hs, w, direction, r_max=8, eps=1e-8)
        J, g = h.grad(torch.tensor(F, device="cuda"), torch.tensor(rec), torch.tensor(d, device="cuda"), 1e-11)
        out[direction] = (J, g.cpu().numpy())
        h.free()
    assert abs(out[1][0] - out[-1][0]) <= 1e-7 * abs(out[1][0])
    g1, g2 = out[1][1], out[-1][1]
    assert np.linalg.norm(g1 - g2) <= 1e-6 * np.linalg.norm(g1)


def test_noalloc_apply_refuses_a_downward_handle(hs):
    w = synth.workload("dir_n127")
    n = w["n"]
    h = _handle(hs, w, -1)
    r = torch.zeros(1, n * n, dtype=torch.complex128, device="cuda")
    z = torch.empty_like(r)
    with pytest.raises(hs.HSweepError):
        hs.hsweep_apply_noalloc(h, r, z)
    h.free()
