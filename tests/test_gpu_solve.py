"""GPU parity of the preconditioned solve (GMRES on M A u = M f, Section 2.4): the
solution against the oracle's direct solve of A u = f, and the GMRES iteration count
against the oracle's H-sweep preconditioned GMRES at the same eps_H and tolerance."""
import numpy as np
import pytest
import torch

import synth
from oracle.assemble import Discretization
from oracle.direct import SparseLU
from oracle.sweep_h import HSweep
from oracle.gmres import preconditioned_solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import paper_1007_4290_gb300 as m
    return m


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_n64_constant_medium_fp64_and_mixed(hs):
    w = synth.workload("n64_const")
    n, omega, pml = w["n"], w["omega"], w["pml"]
    f = w["f"][0].ravel()
    disc = Discretization(w["c"], omega, pml)
    u_ref = SparseLU(disc).solve(f)
    hso = HSweep(disc, w["eps_H"])
    _, it_ref, _ = preconditioned_solve(disc.matrix(), hso.apply, f, w["tol"])
    for prec, tol_err in ((hs.FP64, 1e-6), (hs.MIXED, 1e-5)):
        h = hs.hsweep_setup(torch.tensor(w["c"], device="cuda"), omega, pml, w["eps_H"],
                            hs.default_opts(precision=prec))
        u, it, rr = h.solve(torch.tensor(f, device="cuda")[None], w["tol"])
        err = _rel(u[0].cpu().numpy(), u_ref)
        assert err < tol_err, (prec, err, it, rr)
        if prec == hs.FP64:
            assert abs(it[0] - it_ref) <= 2, (it, it_ref)
        h.free()


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_rhs_and_initial_guess(hs, prec):
    n = 127
    c = synth.velocity_random(n, 1 / 16, 4)
    omega, pml = 2 * np.pi * 8, 10
    pts = synth.source_positions(n, 5, pml, 7)
    F = np.stack([synth.source_delta(n, p).ravel() for p in pts])
    lu = SparseLU(Discretization(c, omega, pml))
    U_ref = np.stack([lu.solve(f) for f in F])
    h = hs.hsweep_setup(torch.tensor(c, device="cuda"), omega, pml, 1e-6, hs.default_opts(precision=prec))
    u, it, rr = h.solve(torch.tensor(F, device="cuda"), 1e-8)
    for s in range(5):
        assert _rel(u[s].cpu().numpy(), U_ref[s]) < (1e-6 if prec == 0 else 1e-5), (s, it, rr)
        assert rr[s] < 1e-5
    # a start from the solution itself needs no iterations
    u0 = torch.tensor(U_ref, device="cuda")
    u2, it2, rr2 = h.solve(torch.tensor(F, device="cuda"), 1e-6, u=u0.clone())
    assert max(it2) == 0 and _rel(u2.cpu().numpy(), U_ref) < 1e-12
    h.free()


def test_iteration_counts_track_the_oracle_h_sweep(hs):
    # FP64 counts within two of the oracle's H-sweep (weak admissibility, same eps_H and
    # GMRES tolerance) at the truncation levels of the workloads
    n = 127
    c = synth.velocity_lens(n)
    omega, pml = 2 * np.pi * 8, 10
    f = synth.source_gaussian(n, (0.5, 0.3), 1 / 32).ravel()
    disc = Discretization(c, omega, pml)
    for eps in (1e-4, 1e-6, 1e-8):
        hso = HSweep(disc, eps, rmax=48)
        _, it_ref, _ = preconditioned_solve(disc.matrix(), hso.apply, f, 1e-8)
        h = hs.hsweep_setup(torch.tensor(c, device="cuda"), omega, pml, eps, hs.default_opts(precision=0))
        _, it, _ = h.solve(torch.tensor(f, device="cuda")[None], 1e-8)
        h.free()
        assert abs(it[0] - it_ref) <= 2, (eps, it, it_ref)


def test_n511_lens_fp64_iteration_count_within_two_of_the_oracle(hs):
    # the workload's size: n = 511, omega / 2 pi = 32, lens, eps_H = 1e-6, rank cap 48;
    # the oracle's H-sweep (Algorithms 2.5/2.6 on the CPU) against the FP64 GPU solve
    w = synth.workload("n511_lens")
    n, omega, pml = w["n"], w["omega"], w["pml"]
    f = w["f"][0].ravel()
    disc = Discretization(w["c"], omega, pml)
    hso = HSweep(disc, w["eps_H"], rmax=48)
    _, it_ref, _ = preconditioned_solve(disc.matrix(), hso.apply, f, w["tol"])
    h = hs.hsweep_setup(torch.tensor(w["c"], device="cuda"), omega, pml, w["eps_H"], hs.default_opts(precision=0))
    _, it, _ = h.solve(torch.tensor(f, device="cuda")[None], w["tol"])
    h.free()
    assert abs(it[0] - it_ref) <= 2, (it, it_ref)


def test_not_converged_is_reported(hs):
    n = 64
    c = synth.velocity_lens(n)
    h = hs.hsweep_setup(torch.tensor(c, device="cuda"), 2 * np.pi * 4, 8, 1e-1,
                        hs.default_opts(precision=0, gmres_max_it=1, refine_max=1))
    f = torch.tensor(synth.source_gaussian(n).ravel(), device="cuda")[None]
    u, it, rr = h.solve(f, 1e-12, check=False)
    code = hs._lib.hsweep_solve(h.raw, hs._ptr(f, torch.complex128), hs._ptr(torch.zeros_like(f), torch.complex128),
                                1, 1e-12, None, None)
    assert code == hs.ERR_NOT_CONVERGED
    assert it[0] == 1
    h.free()


@pytest.mark.parametrize("prec,tol_err", [(1, 1e-5), (0, 1e-6)])
def test_n511_lens_full_size_against_direct_solve(hs, prec, tol_err):
    w = synth.workload("n511_lens")
    n, omega, pml = w["n"], w["omega"], w["pml"]
    f = w["f"][0].ravel()
    u_ref = SparseLU(Discretization(w["c"], omega, pml)).solve(f)
    h = hs.hsweep_setup(torch.tensor(w["c"], device="cuda"), omega, pml, w["eps_H"], hs.default_opts(precision=prec))
    u, it, rr = h.solve(torch.tensor(f, device="cuda")[None], 1e-7)
    err = _rel(u[0].cpu().numpy(), u_ref)
    h.free()
    assert err < tol_err, (err, it, rr)
