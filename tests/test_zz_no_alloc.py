"""hsweep_apply_noalloc: the sweep apply for callers that cannot allocate device memory
(a framework that owns all device memory, a loop where cudaMalloc's implicit
synchronisation is not allowed, an exhausted memory budget).  Its scratch is a fixed
32 MiB device array inside the library instead of on-demand buffers.

It runs the same deterministic kernel as hsweep_apply, so its result must be identical,
on two calls in a row (the array keeps the previous call's contents); the device's free
memory must not change across the call; requests larger than the array are refused.
This file is collected last so that a stop at the first failure has already run every
other test.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


# sweep_kernel 0: the cooperative-team kernel (the automatic choice at these sizes; with
# strong_rank = 2 the sweep on the strongly admissible format); sweep_kernel 1: the basic
# kernel
@pytest.mark.parametrize("n,prec,nrhs,kernel,strong", [(64, 0, 1, 0, 0), (127, 1, 3, 0, 0), (127, 0, 2, 0, 0),
                                                       (127, 1, 2, 1, 0), (64, 0, 3, 1, 0), (127, 0, 2, 0, 2)])
def test_noalloc_apply_matches_apply_twice(n, prec, nrhs, kernel, strong):
    import paper_1007_4290_gb300 as hs
    c = synth.velocity_random(n, 1 / 8, 1)
    omega, pml = 2 * np.pi * (n + 1) / 12, max(2, (n + 1) // 8)
    h = hs.hsweep_setup(torch.tensor(c, device="cuda"), omega, pml, 1e-6,
                        hs.default_opts(precision=prec, sweep_kernel=kernel, strong_rank=strong))
    assert h.sweep_plan(nrhs)["tma"] == (3 if strong else (2 if kernel == 0 else 0))
    for call in range(2):
        r = torch.randn(nrhs, n * n, dtype=torch.complex128, device="cuda")
        ref = h.apply(r)
        z = torch.empty_like(r)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        hs.hsweep_apply_noalloc(h, r, z)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (call, free0, free1)
        assert torch.equal(z, ref), call
    assert h.status()[0] == 0
    h.free()


def test_noalloc_rejects_requests_beyond_the_scratch_array():
    import paper_1007_4290_gb300 as hs
    n = 127
    c = synth.velocity_constant(n)
    h = hs.hsweep_setup(torch.tensor(c, device="cuda"), 2 * np.pi * 8, 10, 1e-6, hs.default_opts(precision=hs.FP64))
    nrhs = hs.NOALLOC_SCRATCH_BYTES // (n * n * 16) + 1       # w cache alone exceeds the array
    r = torch.zeros(nrhs, n * n, dtype=torch.complex128, device="cuda")
    z = torch.empty_like(r)
    code = hs._lib.hsweep_apply_noalloc(h.raw, hs._ptr(r, torch.complex128), hs._ptr(z, torch.complex128), nrhs)
    assert code == hs.ERR_ARG
    assert h.status()[0] == 0
    h.free()
