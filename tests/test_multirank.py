"""The multi-rank paths on CPU with the gloo backend (world size 2): source sharding of the
misfit gradient with its single all-reduce, and the bench's per-rank batches and
max-over-ranks timing."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from oracle import adjoint
from oracle.assemble import Discretization
from oracle.direct import SparseLU


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    n, omega, pml = 23, 2 * np.pi * 2.5, 4
    c_true = synth.velocity_lens(n)
    c = c_true + 0.05 * synth.smooth_noise(n, 1 / 8, 3)
    F = np.stack([synth.source_delta(n, (x, 0.8)).ravel() for x in (0.25, 0.4, 0.55, 0.7, 0.85)])
    rec = (n * 3 // 4) * n + np.arange(n)
    lu = SparseLU(Discretization(c_true, omega, pml))
    d = np.stack([lu.solve(f)[rec] for f in F])
    return c, omega, pml, F, rec, d


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1007_4290_gb300.distributed import sharded_misfit_gradient
        import bench
        c, omega, pml, F, rec, d = _problem()

        def grad_fn(Fl, dl):
            J, g, _ = adjoint.misfit_and_gradient(c, omega, pml, np.asarray(Fl), rec, np.asarray(dl))
            return J, torch.tensor(g.ravel())

        J, g = sharded_misfit_gradient(grad_fn, F, d)
        t = bench.max_over_ranks(10.0 + rank)
        w = synth.workload("n64_const")
        Fr = bench.rank_sources(w, rank)
        out[rank] = (J, g.numpy(), t, Fr)
    finally:
        dist.destroy_process_group()


def test_sharded_gradient_and_bench_rank_logic():
    import __graft_entry__ as ge
    b = ge._build_module()
    if not os.path.exists(b.LIB):
        b.build()
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    c, omega, pml, F, rec, d = _problem()
    J_ref, g_ref, _ = adjoint.misfit_and_gradient(c, omega, pml, F, rec, d)
    for r in range(world):
        J, g, t, Fr = out[r]
        assert abs(J - J_ref) <= 1e-12 * J_ref
        np.testing.assert_allclose(g, g_ref.ravel(), rtol=0, atol=1e-12 * np.max(np.abs(g_ref)))
        assert t == 11.0                      # the job's time is the slowest rank's
        assert Fr.shape == (1, 64 * 64)
    # ranks solve different batches
    assert not np.array_equal(out[0][3], out[1][3])


def _worker_more_ranks_than_sources(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1007_4290_gb300.distributed import sharded_misfit_gradient
        c, omega, pml, F, rec, d = _problem()
        F, d = F[:2], d[:2]

        def grad_fn(Fl, dl):
            J, g, _ = adjoint.misfit_and_gradient(c, omega, pml, np.asarray(Fl), rec, np.asarray(dl))
            return J, torch.tensor(g.ravel())

        J, g = sharded_misfit_gradient(grad_fn, F, d)
        out[rank] = (J, g.numpy(), str(g.device))
    finally:
        dist.destroy_process_group()


def test_sharded_gradient_with_more_ranks_than_sources():
    # world size 3, two sources: one rank owns nothing and still joins the one all-reduce
    # with a buffer on the same device type as the others
    world, port = 3, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker_more_ranks_than_sources, args=(world, port, out), nprocs=world, join=True)
    c, omega, pml, F, rec, d = _problem()
    J_ref, g_ref, _ = adjoint.misfit_and_gradient(c, omega, pml, F[:2], rec, d[:2])
    for r in range(world):
        J, g, dev = out[r]
        assert dev == "cpu"
        assert abs(J - J_ref) <= 1e-12 * J_ref
        np.testing.assert_allclose(g, g_ref.ravel(), rtol=0, atol=1e-12 * np.max(np.abs(g_ref)))


def test_shard_covers_everything_once():
    from paper_1007_4290_gb300.distributed import shard
    for count in (0, 1, 5, 64):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = shard(count, world, r)
                seen += list(range(lo, hi))
                assert hi - lo in (count // world, count // world + 1)
            assert seen == list(range(count))
