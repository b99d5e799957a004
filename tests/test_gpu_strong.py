"""GPU parity of the strongly admissible case (Section 2.3; the configuration of the
experiments of Section 3: R = 2): T~_m is the rank-R projection of the weakly admissible
inverse onto the strong partition (randomized SVD, dense near field), stored exactly in the
sibling-pair factor layout.

Checked against: the exact sweep (dense Algorithm 2.1/2.2 of the oracle) when R is large
enough for the projection to be exact, the expanded-rank formula of the layout, the direct
solve, and the oracle's strong H-sweep iteration counts at R = 2."""
import numpy as np
import pytest
import torch

import synth
from oracle.assemble import Discretization
from oracle.direct import SparseLU
from oracle.gmres import preconditioned_solve
from oracle.hmatrix_strong import Clusters
from oracle.sweep_exact import setup_exact, solve_exact
from oracle.sweep_h import HSweep
from tests.helpers import layer_to_dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import paper_1007_4290_gb300 as m
    return m


def _small():
    n = 31
    c = synth.velocity_random(n, 1 / 8, 0)
    return n, c, 2 * np.pi * 32 / 12.0, 4


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 2e-4)])
def test_strong_form_with_full_rank_is_the_exact_sweep(hs, prec, tol):
    # n = 31, leaves of 8 (depth 2): the well-separated blocks are at most 8 x 8, so
    # R = 8 keeps every singular value and the strong T~_m are the exact T_m
    n, c, omega, pml = _small()
    opts = hs.default_opts(precision=prec, leaf=8, strong_rank=8)
    h = hs.hsweep_setup(torch.tensor(c, device="cuda"), omega, pml, 0.0, opts)
    rng = np.random.default_rng(4)
    R = rng.standard_normal((3, n * n)) + 1j * rng.standard_normal((3, n * n))
    Z = h.apply(torch.tensor(R, device="cuda")).cpu().numpy()
    assert h.status()[0] == 0
    h.free()
    disc = Discretization(c, omega, pml)
    T = setup_exact(disc)
    for s in range(3):
        ref = solve_exact(disc, T, R[s])
        assert np.linalg.norm(Z[s] - ref) / np.linalg.norm(ref) < tol


@pytest.mark.parametrize("R", [1, 2])
def test_well_separated_blocks_of_the_factors_have_rank_at_most_R(hs, R):
    # the strongly admissible structure of every exported T~_m: each block of an
    # interaction list has numerical rank at most R, and the stored sibling ranks stay
    # within 3 R (L - l) + (leaf rows) and within the block dimensions
    w = synth.workload("mixed2_n127")
    n = w["n"]
    opts = hs.default_opts(precision=0, strong_rank=R, pml_sides=w["pml_sides"])
    h = hs.hsweep_setup(torch.tensor(w["c"], device="cuda"), w["omega"], w["pml"], 0.0, opts)
    inf = h.info()
    L = inf["L"]
    ct = Clusters(n, 8)
    assert ct.L == L
    for m in (0, 1, n // 2, n - 1):
        lv, fac, rk = h.export_layer(m)
        for v in range(2, 1 << (L + 1)):
            l = v.bit_length() - 1
            b = v | 1
            leaf_b = (b << (L - l)) - (1 << L)
            cap = min(3 * R * (L - l) + ct.size(L, leaf_b), ct.size(l, (v & ~1) - (1 << l)),
                      ct.size(l, b - (1 << l)))
            assert rk[v] <= cap, (m, v, rk[v], cap)
        T = layer_to_dense(n, 8, inf["r_max"], lv, fac, rk)
        tn = np.linalg.norm(T, 2)
        nblk = 0
        for l in range(2, L + 1):
            for i in range(1 << l):
                for j in ct.interaction_list(l, i):
                    r0, r1 = ct.range(l, i)
                    c0, c1 = ct.range(l, j)
                    sv = np.linalg.svd(T[r0:r1, c0:c1], compute_uv=False)
                    if sv[0] > 1e-6 * tn and sv.size > R:
                        assert sv[R] <= 1e-9 * sv[0], (m, l, i, j, sv[:R + 2])
                        nblk += 1
        assert nblk > 0
    h.free()


@pytest.mark.parametrize("direction", [1, -1])
def test_rank_two_strong_solve_reaches_the_direct_solution(hs, direction):
    # the solve runs on the strong-format sweep (plan kernel 3) in both sweep directions
    w = synth.workload("mixed1_n127")
    n = w["n"]
    disc = Discretization(w["c"], w["omega"], w["pml"], pml_sides=w["pml_sides"])
    f = w["f"].reshape(1, n * n)
    u_ref = SparseLU(disc).solve(f[0])
    for prec in (0, 1):
        opts = hs.default_opts(precision=prec, strong_rank=2, pml_sides=w["pml_sides"], sweep_dir=direction)
        h = hs.hsweep_setup(torch.tensor(w["c"], device="cuda"), w["omega"], w["pml"], 0.0, opts)
        assert h.sweep_plan(1)["tma"] == 3
        u, it, rr = h.solve(torch.tensor(f, device="cuda"), 1e-10)
        h.free()
        u = u.cpu().numpy()[0]
        assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-7, (prec, it)


@pytest.mark.parametrize("name", ["mixed1_n63", "depth1_n63", "dir_n63"])
def test_rank_two_iteration_counts_track_the_oracle_strong_sweep(hs, name):
    # Section 3 protocol: R = 2, GMRES tolerance 1e-3: the GPU's steps within two of the
    # oracle's strong H-sweep
    w = synth.workload(name)
    n = w["n"]
    sides = w.get("pml_sides", 15)
    disc = Discretization(w["c"], w["omega"], w["pml"], pml_sides=sides)
    f = w["f"].reshape(-1).copy()
    if "b_top" in w:
        f += disc.boundary_rhs(3, w["b_top"][0]).ravel()
    S = HSweep(disc, 0.0, leaf=8, rmax=2, admissibility="strong")
    _, it_oracle, _ = preconditioned_solve(disc.matrix(), S.apply, f, 1e-3, 100)
    opts = hs.default_opts(precision=0, strong_rank=2, pml_sides=sides)
    h = hs.hsweep_setup(torch.tensor(w["c"], device="cuda"), w["omega"], w["pml"], 0.0, opts)
    fg = torch.tensor(f.reshape(1, n * n), device="cuda")
    _, it, rr = h.solve(fg, 1e-3)
    h.free()
    assert abs(it[0] - it_oracle) <= 2, (it, it_oracle)


@pytest.mark.parametrize("name", ["pml1_n127", "pml2_n127", "pml3_n127"])
def test_rank_two_counts_on_the_pml_examples_match_the_paper(hs, name):
    # Section 3.1, dependence on omega, at omega / 2 pi = 16 (n + 1 = 128, q = 8, R = 2,
    # tol 1e-3): the paper's tables print 2 GMRES steps for both forces and all three
    # velocity fields; the synthetic fields stand in for the pictured ones, so one step of
    # slack is allowed
    w = synth.workload(name)
    n = w["n"]
    h = hs.hsweep_setup(torch.tensor(w["c"], device="cuda"), w["omega"], w["pml"], 0.0,
                        hs.default_opts(precision=0, strong_rank=2))
    for s in range(2):
        _, it, rr = h.solve(torch.tensor(w["f"][s].reshape(1, n * n), device="cuda"), w["tol"])
        assert it[0] <= 3, (s, it)
    h.free()


@pytest.mark.parametrize("name", ["mixed1_n63", "dir_n63", "depth1_n63"])
@pytest.mark.parametrize("prec", [0, 1])
def test_rank_two_factors_against_the_oracle_strong_factors(hs, name, prec):
    # Section 2.3 (strongly admissible case) at R = 2: the GPU's T~_m and the oracle's strong
    # H-sweep T~_m (F = H.H by the randomized SVD inside every product) against the exact T_m
    # (dense Algorithm 2.1) on the same layers.  The GPU projects an accurate weak inverse
    # onto the strong partition once per layer, so its error is at most the oracle's (20 %
    # slack for the different random test vectors); the two agree with each other to within
    # twice the larger of their errors
    w = synth.workload(name)
    n = w["n"]
    sides = w.get("pml_sides", 15)
    disc = Discretization(w["c"], w["omega"], w["pml"], pml_sides=sides)
    T = setup_exact(disc)
    S = HSweep(disc, 0.0, leaf=8, rmax=2, admissibility="strong")
    opts = hs.default_opts(precision=prec, strong_rank=2, pml_sides=sides)
    h = hs.hsweep_setup(torch.tensor(w["c"], device="cuda"), w["omega"], w["pml"], 0.0, opts)
    rmax = h.info()["r_max"]
    floor = 1e-12 if prec == 0 else 2e-6
    for m in sorted({0, 1, 2, n // 4, n // 2, n - 1}):
        lv, fac, rk = h.export_layer(m)
        Tg = layer_to_dense(n, 8, rmax, lv, fac, rk)
        To = S.T[m].to_dense()
        nx = np.linalg.norm(T[m], 2)
        e_gpu = np.linalg.norm(Tg - T[m], 2) / nx
        e_orc = np.linalg.norm(To - T[m], 2) / nx
        e_both = np.linalg.norm(Tg - To, 2) / nx
        assert e_gpu <= 1.2 * e_orc + floor, (m, e_gpu, e_orc)
        assert e_both <= 2.0 * max(e_gpu, e_orc) + floor, (m, e_both, e_gpu, e_orc)
    h.free()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-5)])
@pytest.mark.parametrize("team,groups,threads", [(0, 0, 0), (1, 4, 0), (2, 4, 0), (4, 2, 0), (8, 1, 0), (16, 8, 0),
                                                 (8, 4, 256), (16, 8, 256)])
def test_strong_format_sweep_matches_the_exact_sweep_of_its_layers(hs, prec, tol, team, groups, threads):
    # the sweep on the strongly admissible format (plan kernel 3) against Algorithm 2.2 of
    # the oracle with every T~_m rebuilt densely from the exported records; n = 127 (L = 4),
    # teams of 1 .. 16 CTAs: no exchange, neighbours only, ancestors at 1 .. 3 depths
    from tests.helpers import strong_to_dense
    if prec == 0 and team == 1:
        pytest.skip("a whole complex128 layer record (two stages) exceeds one CTA's shared memory")
    # FP64: a random smooth medium, eps_H 1e-8 for the weak stage; mixed precision: the
    # converging lens of the paper's PML examples (complex64 setup on the random medium
    # grows T~_m about 25 times by layer 100 and the sweep overflows; FP64 does not)
    if prec == 0:
        n = 127
        c = synth.velocity_random(n, 1 / 8, 1)
        omega, pml, eps = 2 * np.pi * 16, 8, 1e-8
    else:
        w = synth.workload("pml1_n127")
        n, c, omega, pml, eps = w["n"], w["c"], w["omega"], w["pml"], 1e-6
    opts = hs.default_opts(precision=prec, strong_rank=2, team=team, groups=groups, team_threads=threads)
    h = hs.hsweep_setup(torch.tensor(c, device="cuda"), omega, pml, eps, opts)
    nr = 5
    plan = h.sweep_plan(nr)
    assert plan["tma"] == 3 and (threads == 0 or plan["grid_or_threads"] == threads), plan
    rng = np.random.default_rng(7)
    R = rng.standard_normal((nr, n * n)) + 1j * rng.standard_normal((nr, n * n))
    Z = h.apply(torch.tensor(R, device="cuda")).cpu().numpy()
    assert h.status()[0] == 0
    Ts = [strong_to_dense(n, 8, 2, *h.strong_export(m)) for m in range(n)]
    h.free()
    disc = Discretization(c, omega, pml)
    for s in range(nr):
        ref = solve_exact(disc, Ts, R[s])
        assert np.linalg.norm(Z[s] - ref) / np.linalg.norm(ref) < tol, (s, team)


def test_strong_format_records_match_the_stored_expansion(hs):
    # the records hold the strongly admissible T~_m; the sibling-pair store holds the same
    # matrix recompressed to eps_H for the setup's arithmetic
    from tests.helpers import strong_to_dense
    n = 63
    c = synth.velocity_random(n, 1 / 8, 2)
    opts = hs.default_opts(precision=0, strong_rank=2)
    h = hs.hsweep_setup(torch.tensor(c, device="cuda"), 2 * np.pi * 8, 6, 1e-10, opts)
    inf = h.info()
    for m in (0, n // 2, n - 1):
        Ts = strong_to_dense(n, 8, 2, *h.strong_export(m))
        lv, fac, rk = h.export_layer(m)
        Tw = layer_to_dense(n, 8, inf["r_max"], lv, fac, rk)
        assert np.linalg.norm(Ts - Tw) <= 1e-8 * np.linalg.norm(Ts), m
    h.free()


def test_strong_format_sweep_at_n511_matches_the_exact_sweep_of_its_layers(hs):
    # the bench's launch shape (teams of 16 CTAs, 8 RHS per team, several leaves per CTA) at
    # n = 511 on the lens workload in mixed precision, against Algorithm 2.2 of the oracle
    # with the dense T~_m rebuilt from the exported records
    from tests.helpers import strong_to_dense
    w = synth.workload("n511_lens")
    n = w["n"]
    opts = hs.default_opts(precision=1, strong_rank=2, team=16, groups=8)
    h = hs.hsweep_setup(torch.tensor(w["c"], device="cuda"), w["omega"], w["pml"], w["eps_H"], opts)
    nr = 9
    plan = h.sweep_plan(nr)
    assert plan["tma"] == 3 and plan["team_ctas"] == 16 and plan["rhs_per_team"] == 8, plan
    rng = np.random.default_rng(9)
    R = rng.standard_normal((nr, n * n)) + 1j * rng.standard_normal((nr, n * n))
    Z = h.apply(torch.tensor(R, device="cuda")).cpu().numpy()
    assert h.status()[0] == 0
    Ts = [strong_to_dense(n, 8, 2, *h.strong_export(m)) for m in range(n)]
    h.free()
    disc = Discretization(w["c"], w["omega"], w["pml"])
    for s in (0, nr - 1):
        ref = solve_exact(disc, Ts, R[s])
        assert np.linalg.norm(Z[s] - ref) / np.linalg.norm(ref) < 2e-5, s


@pytest.mark.parametrize("R", [1, 3, 5])
def test_strong_format_sweep_for_other_ranks(hs, R):
    # ranks other than the paper's 2: 3R = 3, 9 and 15 columns per cluster (one and two
    # column chunks of the reductions; the expanded store of the setup caps R at 5 here),
    # against Algorithm 2.2 of the oracle with the dense T~_m rebuilt from the exported
    # records
    from tests.helpers import strong_to_dense
    n = 127
    c = synth.velocity_random(n, 1 / 8, 3)
    omega, pml = 2 * np.pi * 12, 8
    opts = hs.default_opts(precision=0, strong_rank=R)
    h = hs.hsweep_setup(torch.tensor(c, device="cuda"), omega, pml, 1e-8, opts)
    nr = 3
    assert h.sweep_plan(nr)["tma"] == 3
    rng = np.random.default_rng(R)
    Rv = rng.standard_normal((nr, n * n)) + 1j * rng.standard_normal((nr, n * n))
    Z = h.apply(torch.tensor(Rv, device="cuda")).cpu().numpy()
    assert h.status()[0] == 0
    Ts = [strong_to_dense(n, 8, R, *h.strong_export(m)) for m in range(n)]
    h.free()
    disc = Discretization(c, omega, pml)
    for s in range(nr):
        ref = solve_exact(disc, Ts, Rv[s])
        assert np.linalg.norm(Z[s] - ref) / np.linalg.norm(ref) < 1e-12, (R, s)
