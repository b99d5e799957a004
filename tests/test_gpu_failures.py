"""Failure handling on the GPU, in the safe forms: every failure is made on the host or
by a wait that nothing satisfies, never by a device fault.

- Allocation failure: the test hook HSWEEP_FAIL_ALLOC_AT fails each device allocation
  of a setup and a solve in turn; every call must return HSWEEP_ERR_OOM, the failed
  setup must hand back no handle, and the device's free memory must come back exactly.
- Zero pivot: a leaf block of A_11 that is exactly singular (c = 1, no PML, omega h = 2,
  a three-row leaf with a zero diagonal) must make the setup return HSWEEP_ERR_NUMERIC.
- Bounded waits: with the test hooks HSWEEP_TEST_WITHHOLD (one CTA of a sweep team never
  publishes its partial sums) and HSWEEP_TEST_WAIT_LIMIT (a short limit on the waits for
  other CTAs' sums), the CTAs that read the withheld sums give up, every CTA returns, the
  status word reads HSWEEP_ERR_TIMEOUT, and the context stays usable.
"""
import os

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import paper_1007_4290_gb300 as m
    return m


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("prec,strong", [(0, 0), (1, 0), (1, 2)])
def test_every_allocation_failure_returns_oom_and_leaks_nothing(hs, prec, strong, monkeypatch):
    # strong = 2: the setup also allocates the projection's plan and scratch and the
    # strongly admissible records, and the solve runs on the strong-format sweep
    w = synth.workload("n64_const")
    n = w["n"]
    c = torch.tensor(w["c"], device="cuda")
    f = torch.tensor(w["f"][0].reshape(1, n * n), device="cuda")
    u = torch.zeros_like(f)
    opts = hs.default_opts(precision=prec, strong_rank=strong)
    # a full run first, so that every kernel module the sequence uses is loaded
    h = hs.hsweep_setup(c, w["omega"], w["pml"], w["eps_H"], opts)
    h.solve(f, 1e-8, u=u)
    h.free()
    k, failures = 1, 0
    while True:
        monkeypatch.setenv("HSWEEP_FAIL_ALLOC_AT", "%d:%d:%d" % (k, prec, strong))
        free0 = _free_bytes()
        code, h = None, None
        try:
            h = hs.hsweep_setup(c, w["omega"], w["pml"], w["eps_H"], opts)
            u.zero_()
            h.solve(f, 1e-8, u=u)
        except hs.HSweepError as e:
            code = e.code
        if h is not None:
            h.free()
        assert _free_bytes() == free0, (k, code)
        if code is None:          # k is past the last allocation of the sequence
            break
        assert code == hs.ERR_OOM, (k, code)
        failures += 1
        k += 1
    monkeypatch.delenv("HSWEEP_FAIL_ALLOC_AT")
    assert failures >= 20, failures
    # the library still works after the failures
    h = hs.hsweep_setup(c, w["omega"], w["pml"], w["eps_H"], opts)
    u.zero_()
    _, it, rr = h.solve(f, 1e-8, u=u)
    h.free()
    assert rr[0] < 1e-6


@pytest.mark.parametrize("prec", [0, 1])
def test_singular_leaf_pivot_is_reported_as_numeric(hs, prec):
    # n = 7, leaves of at most 4 rows: leaves of 4 and 3 rows.  With c = 1, no PML and
    # omega = 2 (n + 1) = 2 / h, every diagonal entry of A_11 is omega^2 - 4 / h^2 = 0
    # (exact in floating point: h = 1/8), so the 3-row leaf is tridiag(64, 0, 64), whose
    # middle eigenvalue 2 * 64 * cos(pi / 2) is zero.
    n = 7
    c = torch.ones(n, n, dtype=torch.float64, device="cuda")
    free0 = _free_bytes()
    with pytest.raises(hs.HSweepError) as e:
        hs.hsweep_setup(c, 2.0 * (n + 1), 0, 1e-8, hs.default_opts(precision=prec, leaf=4))
    assert e.value.code == hs.ERR_NUMERIC
    assert _free_bytes() == free0
    # the same grid at a regular frequency factors and solves
    h = hs.hsweep_setup(c, 2.0 * (n + 1) * 0.77, 0, 1e-8, hs.default_opts(precision=prec, leaf=4))
    f = torch.zeros(1, n * n, dtype=torch.complex128, device="cuda")
    f[0, n * n // 2] = 1.0
    _, it, rr = h.solve(f, 1e-10)
    h.free()
    assert rr[0] < 1e-8


@pytest.mark.parametrize("prec,strong", [(0, 0), (1, 0), (0, 2)])
def test_withheld_partial_sums_time_out_and_every_cta_returns(hs, prec, strong, monkeypatch):
    # strong = 2: the sweep on the strongly admissible format (its partners' sums and the
    # neighbours' boundary rows are what CTA 1 withholds)
    n = 127
    cv = synth.velocity_random(n, 1 / 8, 2)
    omega, pml = 2 * np.pi * 8, 10
    opts = hs.default_opts(precision=prec, team=4, groups=1, strong_rank=strong)
    h = hs.hsweep_setup(torch.tensor(cv, device="cuda"), omega, pml, 1e-6, opts)
    plan = h.sweep_plan(1)
    assert plan["tma"] == (3 if strong else 2) and plan["team_ctas"] == 4, plan
    r = torch.randn(1, n * n, dtype=torch.complex128, device="cuda")
    ref = h.apply(r)
    torch.cuda.synchronize()
    assert h.status()[0] == 0
    monkeypatch.setenv("HSWEEP_TEST_WAIT_LIMIT", "20000")
    monkeypatch.setenv("HSWEEP_TEST_WITHHOLD", "1")       # CTA 1 of team 0
    h.apply(r)                                            # enqueue; the kernel returns
    code, layer = h.status()                              # synchronises
    monkeypatch.delenv("HSWEEP_TEST_WAIT_LIMIT")
    monkeypatch.delenv("HSWEEP_TEST_WITHHOLD")
    assert code == hs.ERR_TIMEOUT and layer >= 0, (code, layer)
    h.free()
    # the context is usable: a new handle applies the same preconditioner again
    h2 = hs.hsweep_setup(torch.tensor(cv, device="cuda"), omega, pml, 1e-6, opts)
    z2 = h2.apply(r)
    torch.cuda.synchronize()
    assert h2.status()[0] == 0
    err = (torch.linalg.norm(z2 - ref) / torch.linalg.norm(ref)).item()
    assert err < (1e-12 if prec == 0 else 1e-5), err
    h2.free()
