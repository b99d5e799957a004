"""GPU parity of the sweep apply (Algorithm 2.6) and of the 5-point matvec.

The apply kernel runs on layers imported from the host in the documented layout;
the reference is the oracle's exact sweep (Algorithm 2.2) run on the dense
matrices those same layers represent, so both sides apply the same T~_m and any
difference is rounding (FP64) or the complex64 arithmetic (mixed)."""
import numpy as np
import pytest
import torch

import synth
from oracle.assemble import Discretization
from oracle.sweep_exact import solve_exact
from tests.helpers import layer_to_dense, random_layer

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import paper_1007_4290_gb300 as m
    return m


def _problem(n, seed):
    c = synth.velocity_random(n, 1 / 8, seed)
    omega = 2 * np.pi * (n + 1) / 12
    return c, omega, max(2, (n + 1) // 8)


def test_matvec_matches_oracle_matrix(hs):
    for n in (17, 64, 127):
        c, omega, pml = _problem(n, 1)
        h = hs.hsweep_create(torch.tensor(c, device="cuda"), omega, pml, 1e-6)
        A = Discretization(c, omega, pml).matrix()
        rng = np.random.default_rng(n)
        X = rng.standard_normal((3, n * n)) + 1j * rng.standard_normal((3, n * n))
        Y = h.matvec(torch.tensor(X, device="cuda")).cpu().numpy()
        ref = (A @ X.T).T
        assert np.linalg.norm(Y - ref) / np.linalg.norm(ref) < 1e-14
        h.free()


def _import_random(hs, h, disc, n, leaf, r_max, seed, full=False, mixed=False):
    # host-made random layers; the reference uses them as the handle stores them (rounded
    # to complex64 on the host in mixed precision), never values read back from the device
    rng = np.random.default_rng(seed)
    scale = 0.3 / np.max(np.abs(disc.north)) / np.sqrt(n)
    dense = []
    for m in range(n):
        lv, fac, rk = random_layer(n, leaf, r_max, rng, scale, full_rank_pairs=full)
        h.import_layer(m, lv, fac, rk)
        if mixed:
            lv = lv.astype(np.complex64).astype(np.complex128)
            fac = fac.astype(np.complex64).astype(np.complex128)
        dense.append(layer_to_dense(n, leaf, r_max, lv, fac, rk))
    rk2 = h.export_layer(n - 1)[2]            # the import/export round trip keeps the ranks
    assert list(rk2[2:]) == list(rk[2:])
    return dense


CASES = [
    # n, precision, team, groups, nrhs
    (64, 0, 1, 1, 1), (64, 0, 8, 1, 1), (64, 0, 8, 2, 3), (37, 0, 4, 4, 5),
    (127, 0, 16, 8, 9), (127, 0, 0, 0, 1), (127, 0, 0, 0, 2), (127, 0, 32, 1, 1),
    (64, 1, 8, 8, 8), (127, 1, 16, 8, 17), (127, 1, 0, 0, 1), (100, 1, 2, 2, 3),
    (255, 0, 32, 1, 1), (255, 0, 0, 0, 1), (255, 1, 32, 2, 2),
]


@pytest.mark.parametrize("n,prec,team,groups,nrhs", CASES)
def test_apply_matches_exact_sweep_on_the_same_layers(hs, n, prec, team, groups, nrhs):
    c, omega, pml = _problem(n, 2)
    disc = Discretization(c, omega, pml)
    leaf, r_max = 8, 12
    opts = hs.default_opts(precision=prec, r_max=r_max, team=team, groups=groups)
    h = hs.hsweep_create(torch.tensor(c, device="cuda"), omega, pml, 1e-6, opts)
    T = _import_random(hs, h, disc, n, leaf, r_max, seed=n + team, mixed=prec == 1)
    rng = np.random.default_rng(7)
    R = rng.standard_normal((nrhs, n * n)) + 1j * rng.standard_normal((nrhs, n * n))
    Z = h.apply(torch.tensor(R, device="cuda")).cpu().numpy()
    assert h.status()[0] == 0
    tol = 1e-12 if prec == 0 else 2e-5
    for s in range(nrhs):
        ref = solve_exact(disc, T, R[s])
        err = np.linalg.norm(Z[s] - ref) / np.linalg.norm(ref)
        assert err < tol, (s, err)
    h.free()


def test_apply_full_rank_blocks_and_repeat_calls_agree(hs):
    n = 64
    c, omega, pml = _problem(n, 3)
    disc = Discretization(c, omega, pml)
    opts = hs.default_opts(precision=0, r_max=32, team=4, groups=2)
    h = hs.hsweep_create(torch.tensor(c, device="cuda"), omega, pml, 1e-6, opts)
    T = _import_random(hs, h, disc, n, 8, 32, seed=11, full=True)
    R = torch.randn(2, n * n, dtype=torch.complex128, device="cuda")
    Z1 = h.apply(R).cpu().numpy()
    Z2 = h.apply(R).cpu().numpy()
    assert np.array_equal(Z1, Z2)           # deterministic reductions
    ref = solve_exact(disc, T, R[1].cpu().numpy())
    assert np.linalg.norm(Z1[1] - ref) / np.linalg.norm(ref) < 1e-12
    h.free()


@pytest.mark.parametrize("n,prec,nrhs,team", [(127, 0, 1, 0), (127, 1, 9, 0), (255, 0, 2, 32), (255, 1, 64, 0),
                                              (64, 1, 3, 4), (37, 0, 2, 0), (255, 1, 17, 0), (255, 0, 5, 0)])
def test_team_sweep_matches_basic_sweep_and_exact(hs, n, prec, nrhs, team):
    # the automatic choice (the cooperative-team kernel) against the basic kernel on the
    # same factors, and against the exact sweep of the exported layers
    c, omega, pml = _problem(n, 4)
    disc = Discretization(c, omega, pml)
    h1 = hs.hsweep_setup(torch.tensor(c, device="cuda"), omega, pml, 1e-6,
                         hs.default_opts(precision=prec, team=team))
    plan = h1.sweep_plan(nrhs)
    assert plan["tma"] == 2, plan
    R = torch.randn(nrhs, n * n, dtype=torch.complex128, device="cuda")
    Z1 = h1.apply(R)
    # the same factors through the basic kernel: rebuild a handle with identical setup
    h2 = hs.hsweep_setup(torch.tensor(c, device="cuda"), omega, pml, 1e-6,
                         hs.default_opts(precision=prec, team=team, sweep_kernel=1))
    Z2 = h2.apply(R)
    torch.cuda.synchronize()
    assert h1.status()[0] == 0 and h2.status()[0] == 0
    tol = 1e-12 if prec == 0 else 2e-5
    err = (torch.linalg.norm(Z1 - Z2) / torch.linalg.norm(Z2)).item()
    assert err < tol, err
    from tests.helpers import layer_to_dense
    T = []
    for m in range(n):
        lv, fac, rk = h1.export_layer(m)
        T.append(layer_to_dense(n, 8, 48, lv, fac, rk))
    ref = solve_exact(disc, T, R[nrhs - 1].cpu().numpy())
    e2 = np.linalg.norm(Z1[nrhs - 1].cpu().numpy() - ref) / np.linalg.norm(ref)
    assert e2 < tol, e2
    h1.free()
    h2.free()


@pytest.mark.parametrize("n,prec,nrhs,team", [(255, 0, 8, 16), (255, 1, 16, 16), (511, 1, 64, 32), (127, 0, 3, 8),
                                              (511, 0, 9, 32)])
def test_two_ctas_per_sm_team_sweep_matches_basic_sweep_and_exact(hs, n, prec, nrhs, team):
    # the 256-thread variant of the team kernel (two CTAs per SM, half the slab rows per
    # CTA) against the basic kernel on the same factors and the exact sweep of the
    # exported layers
    c, omega, pml = _problem(n, 6)
    disc = Discretization(c, omega, pml)
    h1 = hs.hsweep_setup(torch.tensor(c, device="cuda"), omega, pml, 1e-6,
                         hs.default_opts(precision=prec, team=team, team_threads=256))
    plan = h1.sweep_plan(nrhs)
    assert plan["tma"] == 2 and plan["grid_or_threads"] == 256 and plan["team_ctas"] == team, plan
    R = torch.randn(nrhs, n * n, dtype=torch.complex128, device="cuda")
    Z1 = h1.apply(R)
    Z1b = h1.apply(R)
    h2 = hs.hsweep_setup(torch.tensor(c, device="cuda"), omega, pml, 1e-6,
                         hs.default_opts(precision=prec, sweep_kernel=1))
    Z2 = h2.apply(R)
    torch.cuda.synchronize()
    assert h1.status()[0] == 0 and h2.status()[0] == 0
    assert torch.equal(Z1, Z1b)                  # deterministic
    tol = 1e-12 if prec == 0 else 2e-5
    err = (torch.linalg.norm(Z1 - Z2) / torch.linalg.norm(Z2)).item()
    assert err < tol, err
    T = []
    for m in range(n):
        lv, fac, rk = h1.export_layer(m)
        T.append(layer_to_dense(n, 8, 48, lv, fac, rk))
    ref = solve_exact(disc, T, R[nrhs - 1].cpu().numpy())
    e2 = np.linalg.norm(Z1[nrhs - 1].cpu().numpy() - ref) / np.linalg.norm(ref)
    assert e2 < tol, e2
    h1.free()
    h2.free()


@pytest.mark.parametrize("n,nrhs,groups", [(255, 8, 0), (255, 5, 5), (255, 16, 0), (127, 3, 2)])
def test_tensor_core_ancestor_terms_match_cuda_core_path(hs, n, nrhs, groups):
    # complex64 team sweep: ancestor contractions on tensor cores (TF32 in three parts)
    # against the same kernel with every contraction on CUDA cores, and the exact sweep
    c, omega, pml = _problem(n, 5)
    disc = Discretization(c, omega, pml)
    R = torch.randn(nrhs, n * n, dtype=torch.complex128, device="cuda")
    Z = {}
    for tc in (1, 0):
        h = hs.hsweep_setup(torch.tensor(c, device="cuda"), omega, pml, 1e-6,
                            hs.default_opts(precision=1, groups=groups, sweep_tc=tc))
        assert h.sweep_plan(nrhs)["tma"] == 2
        Z[tc] = h.apply(R)
        torch.cuda.synchronize()
        assert h.status()[0] == 0
        if tc == 1:
            T = []
            for m in range(n):
                lv, fac, rk = h.export_layer(m)
                T.append(layer_to_dense(n, 8, 48, lv, fac, rk))
        h.free()
    err = (torch.linalg.norm(Z[1] - Z[0]) / torch.linalg.norm(Z[0])).item()
    assert err < 2e-5, err
    ref = solve_exact(disc, T, R[nrhs - 1].cpu().numpy())
    e2 = np.linalg.norm(Z[1][nrhs - 1].cpu().numpy() - ref) / np.linalg.norm(ref)
    assert e2 < 2e-5, e2


def test_mixed_apply_departs_from_a_linear_map_by_far_less_than_the_solve_assumes(hs):
    # the mixed solve ends its refinement on the inner GMRES estimate once the complex64
    # sweep's departure from linearity (assumed below 1e-5 relative) cannot matter; the
    # departure measured on the n = 511 lens workload must be well below that bound
    w = synth.workload("n511_lens")
    n = w["n"]
    h = hs.hsweep_setup(torch.tensor(w["c"], device="cuda"), w["omega"], w["pml"], w["eps_H"],
                        hs.default_opts(precision=hs.MIXED))
    g = torch.Generator(device="cpu").manual_seed(5)
    X = torch.randn(4, n * n, dtype=torch.complex128, generator=g).cuda()
    Y = 1e-3 * torch.randn(4, n * n, dtype=torch.complex128, generator=g).cuda()
    MX, MY, MXY = h.apply(X), h.apply(Y), h.apply(X + Y)
    torch.cuda.synchronize()
    h.free()
    dev = torch.linalg.norm(MXY - MX - MY, dim=1) / (torch.linalg.norm(MX, dim=1) + torch.linalg.norm(MY, dim=1))
    assert dev.max().item() < 2e-6, dev
