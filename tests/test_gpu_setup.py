"""GPU parity of the setup sweep (Algorithm 2.5): the H-factors T~_m built on the GPU.

Without truncation (eps_H = 0, r_max above every block's size) the H-algebra is exact
(Section 2.3), so every T~_m must equal the dense T_m of the oracle's exact sweep
(Algorithm 2.1).  With truncation the GPU and the oracle's H-sweep are two
approximations of the same T_m; each is compared with T_m, and the apply with the
GPU's own factors is compared element by element with the oracle's exact sweep run
on the very matrices those factors represent."""
import numpy as np
import pytest
import torch

import synth
from oracle.assemble import Discretization
from oracle.sweep_exact import setup_exact, solve_exact
from oracle.sweep_h import HSweep
from tests.helpers import layer_to_dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import paper_1007_4290_gb300 as m
    return m


def _problem(n, seed, ppw=12):
    c = synth.velocity_random(n, 1 / 8, seed)
    omega = 2 * np.pi * (n + 1) / ppw
    return c, omega, max(2, (n + 1) // 8)


def _dense_layers(h, n, leaf, r_max, ms):
    out = {}
    for m in ms:
        lv, fac, rk = h.export_layer(m)
        out[m] = layer_to_dense(n, leaf, r_max, lv, fac, rk)
    return out


@pytest.mark.parametrize("n,prec,tol,core", [(31, 0, 1e-10, 0), (37, 0, 1e-10, 0), (64, 0, 1e-9, 0), (31, 1, 2e-4, 0),
                                          (31, 1, 2e-4, 1), (64, 1, 2e-4, 2), (37, 1, 2e-4, 2)])
def test_setup_without_truncation_is_the_exact_sweep(hs, n, prec, tol, core):
    # core: the recompression cores on the autotuned kernel (0), on CUDA cores (1) or on
    # tensor cores with TF32 operands in three parts (2)
    c, omega, pml = _problem(n, 1)
    disc = Discretization(c, omega, pml)
    T = setup_exact(disc)
    r_max = min(56, (n + 1) // 2)
    h = hs.hsweep_setup(torch.tensor(c, device="cuda"), omega, pml, 0.0,
                        hs.default_opts(precision=prec, r_max=r_max, core_kernel=core))
    assert h.status()[0] == 0
    ms = [0, 1, n // 3, n // 2, n - 1]
    D = _dense_layers(h, n, 8, r_max, ms)
    for m in ms:
        err = np.linalg.norm(D[m] - T[m]) / np.linalg.norm(T[m])
        assert err < tol, (m, err)
    h.free()


@pytest.mark.parametrize("prec", [0, 1])
def test_setup_with_truncation_approximates_T_like_the_oracle(hs, prec):
    n, eps = 63, 1e-6
    c, omega, pml = _problem(n, 2)
    disc = Discretization(c, omega, pml)
    T = setup_exact(disc)
    hso = HSweep(disc, eps)
    h = hs.hsweep_setup(torch.tensor(c, device="cuda"), omega, pml, eps, hs.default_opts(precision=prec))
    ms = [0, n // 4, n // 2, n - 1]
    D = _dense_layers(h, n, 8, 48, ms)
    for m in ms:
        e_gpu = np.linalg.norm(D[m] - T[m]) / np.linalg.norm(T[m])
        e_ora = np.linalg.norm(hso.T[m].to_dense() - T[m]) / np.linalg.norm(T[m])
        assert e_gpu < (2e-5 if prec == 0 else 2e-4), (m, e_gpu, e_ora)
        # ranks of the top blocks within a few of the oracle's
        rk = h.layer_ranks(m)
        ro = hso.ranks(m)
        assert abs(rk[2] - ro[1][0]) <= 3, (m, rk[2], ro[1])
    h.free()


@pytest.mark.parametrize("n,prec,nrhs", [(63, 0, 1), (64, 0, 3), (127, 1, 4)])
def test_apply_with_gpu_factors_matches_exact_sweep_on_them(hs, n, prec, nrhs):
    c, omega, pml = _problem(n, 3)
    disc = Discretization(c, omega, pml)
    h = hs.hsweep_setup(torch.tensor(c, device="cuda"), omega, pml, 1e-6, hs.default_opts(precision=prec))
    D = _dense_layers(h, n, 8, 48, range(n))
    T = [D[m] for m in range(n)]
    rng = np.random.default_rng(5)
    R = rng.standard_normal((nrhs, n * n)) + 1j * rng.standard_normal((nrhs, n * n))
    Z = h.apply(torch.tensor(R, device="cuda")).cpu().numpy()
    for s in range(nrhs):
        ref = solve_exact(disc, T, R[s])
        err = np.linalg.norm(Z[s] - ref) / np.linalg.norm(ref)
        assert err < (1e-11 if prec == 0 else 1e-4), (s, err)
    h.free()


def test_core_product_autotuning_reports_its_choice(hs):
    # complex64: the setup times the CUDA-core and tensor-core kernels of the recompression
    # cores on its middle layer and keeps the faster; complex128 always uses CUDA cores
    w = synth.workload("n511_lens")
    c = torch.tensor(w["c"], device="cuda")
    h = hs.hsweep_setup(c, w["omega"], w["pml"], w["eps_H"], hs.default_opts(precision=hs.MIXED))
    t = h.setup_tuning()
    h.free()
    assert t["per_layer"] in (0, 1), t
    assert all(x > 0 for x in t["ms"][1]), t
    assert t["per_layer"] == (1 if t["ms"][1][1] < t["ms"][1][0] else 0)
    h = hs.hsweep_setup(c[:64, :64].contiguous(), 2 * np.pi * 4, 8, 1e-6, hs.default_opts(precision=hs.FP64))
    assert h.setup_tuning()["per_layer"] == -1
    h.free()
