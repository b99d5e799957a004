"""The sweep apply (Algorithm 2.6) captured into a CUDA graph and replayed.

For an upward handle hsweep_apply enqueues one memset of the exchange slots and one
cooperative sweep launch on the handle's stream, so once the handle's buffers are large
enough the call can be captured; hsweep_apply_noalloc can be captured at any time.  The
kernels are deterministic, so a replay must give exactly the eager result for the current
contents of r, for every sweep kernel (the cooperative teams in both precisions, the basic
kernel, the strongly admissible records).  A capture that would have to allocate, or of a
downward handle, is refused; buffers outgrown after a capture stay valid for the graph.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import paper_1007_4290_gb300 as m
    return m


def _setup(hs, n, **opts):
    c = torch.tensor(synth.velocity_random(n, 1 / 8, 1), device="cuda")
    omega, pml = 2 * np.pi * (n + 1) / 12, max(2, (n + 1) // 8)
    return hs.hsweep_setup(c, omega, pml, 1e-6, hs.default_opts(**opts))


def _raw_apply(hs, fn, h, r, z):
    return fn(h.raw, hs._ptr(r, torch.complex128), hs._ptr(z, torch.complex128), r.shape[0])


# (precision, sweep_kernel, strong_rank, nrhs, entry point, expected plan): plan 2 the
# cooperative-team kernel, 0 the basic kernel, 3 the strongly admissible records
@pytest.mark.parametrize("prec,kernel,strong,nrhs,noalloc,plan", [
    (1, 0, 0, 8, False, 2), (0, 0, 0, 2, False, 2), (1, 1, 0, 3, False, 0),
    (1, 0, 2, 8, False, 3), (1, 0, 0, 2, True, 2), (0, 0, 2, 2, True, 3)])
def test_graph_replay_equals_the_eager_apply(hs, prec, kernel, strong, nrhs, noalloc, plan):
    n = 127
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        h = _setup(hs, n, precision=prec, sweep_kernel=kernel, strong_rank=strong)
        assert h.sweep_plan(nrhs)["tma"] == plan
        r = torch.randn(nrhs, n * n, dtype=torch.complex128, device="cuda")
        z = torch.zeros_like(r)
        h.apply(r)                       # sizes the handle's buffers outside the capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    fn = hs._lib.hsweep_apply_noalloc if noalloc else hs._lib.hsweep_apply
    with torch.cuda.graph(g, stream=s):
        code = _raw_apply(hs, fn, h, r, z)
    assert code == hs.OK
    for k in range(3):
        with torch.cuda.stream(s):
            if k:
                r.copy_(torch.randn_like(r))
            ref = h.apply(r)
            z.zero_()
            g.replay()
        s.synchronize()
        assert torch.equal(z, ref), k
    assert h.status()[0] == 0
    del g
    h.free()


def test_capture_that_needs_larger_buffers_is_refused(hs):
    n = 63
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        h = _setup(hs, n, precision=hs.MIXED)
        r = torch.randn(4, n * n, dtype=torch.complex128, device="cuda")
        z = torch.zeros_like(r)
        h.apply(r[:1])                   # buffers for one right-hand side only
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        code = _raw_apply(hs, hs._lib.hsweep_apply, h, r, z)
    assert code == hs.ERR_ARG
    del g
    # the handle is unharmed: the same call outside a capture works
    with torch.cuda.stream(s):
        z2 = h.apply(r)
    s.synchronize()
    assert torch.isfinite(torch.view_as_real(z2)).all()
    assert h.status()[0] == 0
    h.free()


def test_buffers_outgrown_after_a_capture_stay_valid_for_the_graph(hs):
    n = 63
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        h = _setup(hs, n, precision=hs.MIXED)
        r = torch.randn(2, n * n, dtype=torch.complex128, device="cuda")
        z = torch.zeros_like(r)
        h.apply(r)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        assert _raw_apply(hs, hs._lib.hsweep_apply, h, r, z) == hs.OK
    with torch.cuda.stream(s):
        big = torch.randn(12, n * n, dtype=torch.complex128, device="cuda")
        zb = h.apply(big)                # outgrows the w cache the graph points into
        ref = h.apply(r)
        g.replay()
    s.synchronize()
    assert torch.equal(z, ref)
    assert torch.isfinite(torch.view_as_real(zb)).all()
    assert h.status()[0] == 0
    del g
    h.free()


def test_capture_of_a_downward_handle_is_refused(hs):
    n = 63
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        h = _setup(hs, n, precision=hs.MIXED, sweep_dir=-1)
        r = torch.randn(1, n * n, dtype=torch.complex128, device="cuda")
        z = torch.zeros_like(r)
        h.apply(r)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        code = _raw_apply(hs, hs._lib.hsweep_apply, h, r, z)
    assert code == hs.ERR_ARG
    del g
    h.free()
