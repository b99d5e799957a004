"""Benchmark: preconditioned Helmholtz solves per second on one GB300 (or N, weak scaling).

Workload (default): n = 1023 (N = 1,046,529 unknowns), omega/2pi = 64, random smooth
velocity c = 1 + 0.2 g (filter width 1/32, seed 1), PML 16 cells, 64 point sources at
seeded positions, eps_H = 1e-6, mixed precision (complex64 H-factors and sweeps, FP64
GMRES and refinement), all 64 right-hand sides in one batched solve.

A step is one batched preconditioned solve of the 64 right-hand sides (GMRES on
M A u = M f with the sweep apply of Algorithm 2.6 inside); the setup sweep
(Algorithm 2.5) runs once before the timed region and is reported as setup_s.
value = right-hand sides solved per second (to ||M(f - A u)|| <= tol ||M f||, which
the parity tests tie to a relative error <= 1e-5 against the direct solve).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--fp64]

Under torchrun every rank builds its own factorisation (a replica) and solves its
own batch of 64 sources; there is no collective on the data path.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "n1023_random"
METRIC = "preconditioned solves/sec at n=1023 (mixed vs FP64, rel err 1e-6); setup s"
SOLVE_TOL = 1e-7


def _tree_sizes(n, leaf=8):
    L = 0
    while -(-n // (1 << L)) > leaf:
        L += 1
    nn = 1 << (L + 1)
    sz = [0] * nn
    sz[1] = n
    for v in range(1, nn // 2):
        a = (sz[v] + 1) // 2
        sz[2 * v], sz[2 * v + 1] = a, sz[v] - a
    return L, sz


def sweep_work(h, n, nrhs, elem_bytes):
    """Algorithmic flops and HBM bytes of one sweep launch (Algorithm 2.6 over nrhs RHS).
    Per layer step: leaves sz^2 complex MACs per RHS, every factor entry used twice
    (reduction F^t x and expansion F q) per RHS; the factors are read once per step."""
    L, sz = _tree_sizes(n)
    leaf_e = sum(sz[v] * sz[v] for v in range(1 << L, 1 << (L + 1)))
    lr = []
    for m in range(n):
        rk = h.layer_ranks(m)
        lr.append(sum(sz[v] * rk[v] for v in range(2, 1 << (L + 1))))
    steps = list(range(n)) + list(range(n - 1))      # forward layers, then backward layers
    macs = sum(leaf_e + 2 * lr[m] for m in steps)
    flops = 8.0 * nrhs * macs
    fac_bytes = sum(leaf_e + lr[m] for m in steps) * elem_bytes
    vec_bytes = nrhs * n * n * (16 + 16 + 2 * elem_bytes)   # read r, write z, w written + read
    return flops, fac_bytes + vec_bytes, sum(lr) + n * leaf_e


# DRAM bytes (read + write) of one sweep launch, from ncu captures summarised in profiles/,
# keyed by workload and right-hand sides, with the SHA-256 of the kernel source they were
# taken on: a changed kernel reports null instead of a stale number.
SWEEP_TRAFFIC = {
    # profiles/sweep_team_n1023_random_64rhs_dram.md: 3.97 GB read + 1.57 GB written
    "n1023_random/64": {"sha256": "75467c6fcf28dfa9fd94fa0d13c92a263363a102bddc6ec57678f988fd9e60fa",
                        "bytes": 5.54e9},
}
TEAM_KERNEL_SRC = os.path.join(ROOT, "paper_1007_4290_gb300", "csrc", "sweep_team.cu")


def recorded_traffic(workload, nrhs):
    rec = SWEEP_TRAFFIC.get("%s/%d" % (workload, nrhs))
    if rec is None or not os.path.exists(TEAM_KERNEL_SRC):
        return None
    import hashlib
    with open(TEAM_KERNEL_SRC, "rb") as fh:
        digest = hashlib.sha256(fh.read()).hexdigest()
    return rec["bytes"] if digest == rec["sha256"] else None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                for line in out.stdout.strip().splitlines():
                    self.rows.append([x.strip() for x in line.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def fp32_alu_peak_tflops():
    """FP32 FMA peak from the unit counts: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz."""
    return 152 * 128 * 2 * 2.07e9 / 1e12


# ---------------------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on a bounded sample of the same workload.
def cpu_sample(budget_s, applies_per_solve, n_layers_cap=None):
    """Times the oracle's Algorithm 2.5 setup and Algorithm 2.6 apply on the first
    layers of the workload until about budget_s of work, and scales the per-layer
    apply time to the full sweep (2n - 1 layer steps).  Runs single-threaded."""
    from oracle.assemble import Discretization
    from oracle.hmatrix import Trunc, hinv, hsub, tree_depth
    from oracle.sweep_h import tridiag_H
    w = synth.workload(WORKLOAD)
    disc = Discretization(w["c"], w["omega"], w["pml"])
    n = disc.n
    tr = Trunc(w["eps_H"], 48)
    L = tree_depth(n, 8)
    T = []
    t0 = time.perf_counter()
    m = 0
    while m < n and (time.perf_counter() - t0 < 0.6 * budget_s or m < 3):
        if n_layers_cap is not None and m >= n_layers_cap:
            break
        Amm = tridiag_H(disc.diag[m], disc.east[m, 1:-1], 0, 0, L)
        S = Amm if m == 0 else hsub(Amm, T[m - 1].diagmul(dl=disc.A_off(m), dr=disc.A_off(m)), tr)
        T.append(hinv(S, tr))
        m += 1
    t_setup = time.perf_counter() - t0
    ms = len(T)
    f = w["f"][0].reshape(n, n)
    u = f[:ms].copy()
    t1 = time.perf_counter()
    wv = []
    for k in range(ms):                       # forward steps on the sampled layers
        wv.append(T[k].matvec(u[k]))
        if k + 1 < ms:
            u[k + 1] = u[k + 1] - disc.A_off(k + 1) * wv[k]
    for k in range(ms - 2, -1, -1):           # backward steps
        u[k] = wv[k] - T[k].matvec(disc.A_off(k + 1) * u[k + 1])
    t_apply = time.perf_counter() - t1
    per_step = t_apply / (2 * ms - 1)
    t_solve = applies_per_solve * per_step * (2 * n - 1)
    return {"value": 1.0 / t_solve, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": "oracle H-sweep (Algorithms 2.5/2.6, eps_H 1e-6) on the first %d of %d layers: "
                      "setup %.1f s, %.1f ms per layer step; per-solve time = %.2f applies x %d layer steps"
                      % (ms, n, t_setup, 1e3 * per_step, applies_per_solve, 2 * n - 1),
            "setup_s_extrapolated": t_setup / ms * n, "seconds": t_setup + t_apply}


def run_cpu_sample_subprocess(budget_s, applies_per_solve):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", str(budget_s),
                          str(applies_per_solve)], capture_output=True, text=True, env=env, timeout=600)
    for line in out.stdout.splitlines()[::-1]:
        if line.startswith("{"):
            return json.loads(line)
    raise RuntimeError("cpu sample failed: " + out.stderr[-2000:])


# ---------------------------------------------------------------------------------------
def rank_sources(w, rank):
    """The batch of right-hand sides of one rank, (nrhs, n*n): rank 0 solves the workload's
    own sources, every other rank the same number of point sources at its own seed."""
    n, pml, F = w["n"], w["pml"], w["f"]
    if rank > 0:
        pts = synth.source_positions(n, F.shape[0], pml, 100 + rank)
        F = np.stack([synth.source_delta(n, p) for p in pts])
    return F.reshape(F.shape[0], n * n)


def max_over_ranks(ms, device=None):
    """Largest value over the ranks of the default process group (the job's time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64", action="store_true", help="also time the FP64 sweep (nrhs = 1 per call)")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--cpu-sample", nargs=2, default=None)
    ap.add_argument("--workload", default=WORKLOAD,
                    help="synthetic workload (n1023_random, n511_lens, n64_const, n2047_random)")
    ap.add_argument("--apply-only", type=int, default=0, metavar="NRHS",
                    help="time only the sweep apply (Algorithm 2.6) on NRHS right-hand sides")
    ap.add_argument("--setup-only", action="store_true", help="time only the setup sweep (Algorithm 2.5)")
    ap.add_argument("--team", type=int, default=0, help="with --apply-only: CTAs per sweep team (0 = automatic)")
    ap.add_argument("--groups", type=int, default=0, help="with --apply-only: right-hand sides per team (0 = automatic)")
    ap.add_argument("--sweep-tc", type=int, default=0, help="with --apply-only: ancestor contractions on tensor cores")
    ap.add_argument("--boundary-table", default="",
                    help="comma-separated n: GMRES steps and times of the boundary-condition examples of "
                         "Section 3.2 (depth extrapolation, mixed PML / Dirichlet), one JSON line")
    ap.add_argument("--direction-table", default="",
                    help="comma-separated n (e.g. 127,255,511): GMRES steps and times of the upward and "
                         "downward sweeps on the sweeping-direction workload (Section 3.1), one JSON line")
    ap.add_argument("--pml-table", default="",
                    help="comma-separated n: GMRES steps and times of the PML examples of Section 3.1 "
                         "(lens, waveguide, random medium; point source and wave packet), one JSON line")
    ap.add_argument("--q-table", default="",
                    help="comma-separated n (255,511,1023,2047 for q = 8..64): the PML examples at omega / 2 pi = 32 "
                         "(Section 3.1, dependence on q), one JSON line")
    ap.add_argument("--fields", default="1,2,3", help="with --pml-table / --q-table: velocity fields (1 lens, "
                                                       "2 waveguide, 3 random medium)")
    ap.add_argument("--strong-rank", type=int, default=0,
                    help="with --direction-table / --boundary-table / --pml-table / --apply-only / --setup-only: "
                         "strongly admissible H-matrices of "
                         "rank R (Section 2.3; Section 3 uses R = 2) instead of weak ones of rank 2")
    args = ap.parse_args()

    if args.cpu_sample is not None:
        print(json.dumps(cpu_sample(float(args.cpu_sample[0]), float(args.cpu_sample[1]))))
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.direction_table:
        run_direction_table(args)
        return
    if args.pml_table or args.q_table:
        run_pml_table(args)
        return
    if args.boundary_table:
        run_boundary_table(args)
        return
    if args.apply_only or args.setup_only:
        run_parts(args)
        return

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1007_4290_gb300 as hs

    w = synth.workload(args.workload)
    n, omega, pml, eps = w["n"], w["omega"], w["pml"], w["eps_H"]
    F = rank_sources(w, rank)
    nrhs = F.shape[0]
    dev = torch.device("cuda", local)
    c_d = torch.tensor(w["c"], device=dev)
    f_d = torch.tensor(F, device=dev)
    u_d = torch.zeros_like(f_d)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # setup (Algorithm 2.5), once
    barrier()
    t0 = time.perf_counter()
    h = hs.hsweep_setup(c_d, omega, pml, eps, hs.default_opts(precision=hs.MIXED))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    info = h.info()

    def step(u):
        u.zero_()
        _, it, rr = h.solve(f_d, SOLVE_TOL, u=u)
        return it, rr

    for _ in range(max(3, args.warmup)):
        it, rr = step(u_d)
    # L2: the 1 GB right-hand-side batch and the factors (GBs) exceed the 129 MB L2
    h.stats(reset=True)
    h.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            it, rr = step(u_d)
        e1.record(stream)
        barrier()
    h.profile(False)
    launches, sweeps, sweep_ms = h.stats(reset=True)
    ms = e0.elapsed_time(e1)
    t_max = max_over_ranks(ms, dev if world > 1 else None)
    total_solves = nrhs * args.steps * world
    value = total_solves / (t_max / 1e3)

    # end to end through the public API with host buffers (pinned), every step's copies
    # inside the timed region.  Serial: H2D, solve, D2H, host sync per step.  Pipelined (the
    # reported e2e): two device buffers; on a copy stream the inputs of step i+1 are
    # uploaded while step i solves, and the result of step i is read back while step i+1
    # solves (the copy engines run beside the kernels).
    f_h = torch.tensor(F).pin_memory()
    u_h = [torch.empty_like(f_h).pin_memory() for _ in range(2)]
    f_dd = [f_d, torch.empty_like(f_d)]
    u_dd = [u_d, torch.empty_like(u_d)]
    cstream = torch.cuda.Stream(device=dev)

    def step_serial():
        f_d.copy_(f_h, non_blocking=True)
        step(u_d)
        u_h[0].copy_(u_d, non_blocking=True)
        stream.synchronize()        # the host holds the step's result before the next step

    def run_pipelined(k):
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        with torch.cuda.stream(cstream):
            f_dd[0].copy_(f_h, non_blocking=True)
        ev_in[0].record(cstream)
        for i in range(k):
            b = i % 2
            stream.wait_event(ev_in[b])
            if i + 1 < k:
                # buffer 1-b was last read by step i-1, which hsweep_solve completed
                with torch.cuda.stream(cstream):
                    f_dd[1 - b].copy_(f_h, non_blocking=True)
                ev_in[1 - b].record(cstream)
            step(u_dd[b])           # returns after the step's kernels finished
            ev_done[b].record(stream)
            cstream.wait_event(ev_done[b])
            with torch.cuda.stream(cstream):
                u_h[b].copy_(u_dd[b], non_blocking=True)
        cstream.synchronize()       # the host holds every step's result

    def timed(fn, k):
        barrier()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(cstream)
        stream.wait_event(ea)
        fn(k)
        cstream.wait_stream(stream)
        eb.record(cstream)
        barrier()
        return max_over_ranks(ea.elapsed_time(eb), dev if world > 1 else None)

    for _ in range(2):
        step_serial()
    ms_serial = timed(lambda k: [step_serial() for _ in range(k)], args.steps)
    run_pipelined(2)
    ms_e2e = timed(run_pipelined, args.steps)
    e2e_value = total_solves / (ms_e2e / 1e3)
    e2e_serial = total_solves / (ms_serial / 1e3)

    # roofline of the dominant kernel (the sweep apply), from the live CUDA-event timing
    flops, bytes_, stored = sweep_work(h, n, nrhs, info["bytes_per_entry"])
    avg_s = (sweep_ms / max(1, sweeps)) / 1e3
    peaks, src = _peaks()
    alu_peak = fp32_alu_peak_tflops()
    t_alu = flops / (alu_peak * 1e12)
    t_hbm = bytes_ / (peaks["hbm_gbs"] * 1e9)
    if t_alu >= t_hbm:
        roof = {"bound": "alu", "achieved": flops / avg_s / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
                "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 x 2.07 GHz (unit counts)"}
    else:
        roof = {"bound": "hbm", "achieved": bytes_ / avg_s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "peak_source": src}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = recorded_traffic(args.workload, nrhs)
    plan = h.sweep_plan(nrhs)
    roof["kernel"] = {2: "sweep_team_kernel", 1: "sweep_tma_kernel"}.get(plan["tma"], "sweep_kernel") + "<c64>"
    roof["plan"] = plan
    roof["launch_ms"] = avg_s * 1e3
    roof["hbm_gbs_achieved"] = bytes_ / avg_s / 1e9
    roof["hbm_frac"] = roof["hbm_gbs_achieved"] / peaks["hbm_gbs"]
    roof["algorithmic_flops_per_launch"] = flops
    roof["algorithmic_bytes_per_launch"] = bytes_

    fp64 = None
    if args.fp64:
        t0 = time.perf_counter()
        h64 = hs.hsweep_setup(c_d, omega, pml, eps, hs.default_opts(precision=hs.FP64))
        torch.cuda.synchronize()
        s64 = time.perf_counter() - t0
        u1 = torch.zeros_like(f_d[:1])
        h64.solve(f_d[:1], SOLVE_TOL, u=u1)
        k64 = 4
        torch.cuda.synchronize()
        e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e4.record(stream)
        its = []
        for s in range(k64):
            u1.zero_()
            _, it1, _ = h64.solve(f_d[s:s + 1], SOLVE_TOL, u=u1)
            its.append(it1[0])
        e5.record(stream)
        torch.cuda.synchronize()
        fp64 = {"solves_per_s": k64 / (e4.elapsed_time(e5) / 1e3), "setup_s": s64, "nrhs_per_call": 1,
                "gmres_iters": its}
        h64.free()

    cpu = None
    if rank == 0 and world == 1:
        applies = sweeps / max(1, args.steps)
        try:
            cpu = run_cpu_sample_subprocess(args.cpu_budget, applies)
        except Exception as e:  # the baseline is reported, never required
            cpu = {"error": str(e)[:200]}
    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64 factors+sweeps / f64 Krylov",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "N": n * n, "omega_over_2pi": omega / (2 * np.pi),
                       "pml": pml, "eps_H": eps, "nrhs": nrhs, "precision": "mixed", "tol": SOLVE_TOL,
                       "parallelism": "replica per GPU, sources sharded" if world > 1 else "1 GPU",
                       "l2": "inputs larger than L2 (1 GB RHS batch, factors %.2f GB)" % (
                           stored * info["bytes_per_entry"] / 1e9)},
            "setup_s": setup_s,
            "gmres_iters": {"min": min(it), "max": max(it), "mean": float(np.mean(it))},
            "relres_max": max(rr),
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": int(f_h.numel() * 16),
                    "d2h_bytes_per_step": int(u_h[0].numel() * 16),
                    "transfers": "pinned host buffers; inputs of step i+1 uploaded and results of step i read "
                                 "back on a copy stream while the solves run (two device buffers)",
                    "serial_value": e2e_serial},
            "gpu_launches": launches,
            "sweep_launches_per_step": sweeps / args.steps,
            "roofline": roof,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        if fp64 is not None:
            line["fp64"] = fp64
            line["mixed_over_fp64"] = value / fp64["solves_per_s"]
        print(json.dumps(line))
    h.free()
    if world > 1:
        dist.destroy_process_group()


def _rank_opts(args, w):
    """Options of the paper-protocol tables: FP64 with R = 2 on the weakly admissible blocks,
    or with --strong-rank R the strongly admissible case (the configuration of Section 3),
    in mixed precision: its weak inverse runs at the default rank cap with eps_H = 1e-6
    before the rank-R projection (FP64 at that cap would take minutes per setup at n = 1023)."""
    import paper_1007_4290_gb300 as hs
    if args.strong_rank > 0:
        return {"strong_rank": args.strong_rank, "precision": hs.MIXED}, 1e-6
    return {"r_max": w["r_max"], "precision": hs.FP64}, w["eps_H"]


def _rank_label(args):
    if args.strong_rank > 0:
        return "mixed precision, strong admissibility, R = %d" % args.strong_rank
    return "FP64, weak admissibility, R = 2"


def run_direction_table(args):
    """The sweeping-direction test of Section 3.1 (c = 1/2 + x2, point source at
    (0.125, 0.5), q = 8, fixed rank R = 2, GMRES tolerance 1e-3, FP64): setup and solve
    times and GMRES steps of the upward (+x2) and downward (-x2) sweeps, per n."""
    import torch
    import paper_1007_4290_gb300 as hs
    rows = []
    for n in [int(v) for v in args.direction_table.split(",")]:
        w = synth.workload("dir_n%d" % n)
        f = torch.tensor(w["f"].reshape(1, -1), device="cuda")
        row = {"n": n, "omega_over_2pi": w["omega"] / (2 * np.pi), "R": w["r_max"]}
        for direction, key in ((1, "up"), (-1, "down")):
            kw, eps = _rank_opts(args, w)
            opts = hs.default_opts(sweep_dir=direction, **kw)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = hs.hsweep_setup(torch.tensor(w["c"], device="cuda"), w["omega"], w["pml"], eps, opts)
            torch.cuda.synchronize()
            t_setup = time.perf_counter() - t0
            u = torch.zeros_like(f)
            h.solve(f, w["tol"], u=u, check=False)
            u.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, it, rr = h.solve(f, w["tol"], u=u, check=False)
            torch.cuda.synchronize()
            row[key] = {"setup_s": t_setup, "solve_s": time.perf_counter() - t0, "iters": it[0], "relres": rr[0]}
            h.free()
        rows.append(row)
    print(json.dumps({"metric": "GMRES steps, sweeping-direction test (Section 3.1), %s, tol 1e-3"
                                % _rank_label(args), "data": "synthetic", "rows": rows}))


def run_boundary_table(args):
    """The boundary-condition examples of Section 3.2 (q = 8, fixed rank R = 2, tol 1e-3,
    FP64, upward sweep): depth extrapolation in a waveguide with Dirichlet data on x2 = 1
    (b = 1 and a slant wave), and c = 1 with zero Dirichlet on x1 = 0, 1 (mixed1) or on
    x1 = 1 and x2 = 1 (mixed2), a PML on the other sides."""
    import torch
    import paper_1007_4290_gb300 as hs
    rows = []
    for n in [int(v) for v in args.boundary_table.split(",")]:
        row = {"n": n}
        for kind in ("depth1", "depth2", "mixed1", "mixed2"):
            w = synth.workload("%s_n%d" % (kind, n))
            kw, eps = _rank_opts(args, w)
            opts = hs.default_opts(pml_sides=w["pml_sides"], **kw)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = hs.hsweep_setup(torch.tensor(w["c"], device="cuda"), w["omega"], w["pml"], eps, opts)
            torch.cuda.synchronize()
            t_setup = time.perf_counter() - t0
            f0 = torch.tensor(w["f"].reshape(1, -1), device="cuda")
            if "b_top" in w:
                h.boundary_rhs(3, torch.tensor(w["b_top"], device="cuda"), f0)
            u = torch.zeros_like(f0)
            h.solve(f0, w["tol"], u=u, check=False)
            u.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, it, rr = h.solve(f0, w["tol"], u=u, check=False)
            torch.cuda.synchronize()
            row[kind] = {"setup_s": t_setup, "solve_s": time.perf_counter() - t0, "iters": it[0], "relres": rr[0]}
            h.free()
        rows.append(row)
    print(json.dumps({"metric": "GMRES steps, boundary-condition examples (Section 3.2), %s, tol 1e-3"
                                % _rank_label(args), "data": "synthetic", "rows": rows}))


def run_pml_table(args):
    """The dependence-on-omega tables of Section 3.1 (PML on all sides; the lens, the
    waveguide and a random medium; a point source and a wave packet; q = 8, R = 2,
    tol 1e-3): setup time, and GMRES steps and solve time per force, per n."""
    import torch
    import paper_1007_4290_gb300 as hs
    rows = []
    sizes = args.pml_table or args.q_table
    prefix = "pml" if args.pml_table else "qpml"
    for n in [int(v) for v in sizes.split(",")]:
        for kind in ["%s%s" % (prefix, k) for k in args.fields.split(",")]:
            w = synth.workload("%s_n%d" % (kind, n))
            kw, eps = _rank_opts(args, w)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = hs.hsweep_setup(torch.tensor(w["c"], device="cuda"), w["omega"], w["pml"], eps, hs.default_opts(**kw))
            torch.cuda.synchronize()
            row = {"n": n, "field": kind, "setup_s": time.perf_counter() - t0}
            for s, key in ((0, "point"), (1, "packet")):
                f = torch.tensor(w["f"][s].reshape(1, -1), device="cuda")
                u = torch.zeros_like(f)
                h.solve(f, w["tol"], u=u, check=False)
                u.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, it, rr = h.solve(f, w["tol"], u=u, check=False)
                torch.cuda.synchronize()
                row[key] = {"iters": it[0], "solve_s": time.perf_counter() - t0, "relres": rr[0]}
            h.free()
            rows.append(row)
    what = "dependence on omega, q = 8" if args.pml_table else "dependence on q, omega / 2 pi = 32"
    print(json.dumps({"metric": "GMRES steps, PML examples (Section 3.1, %s), %s, tol 1e-3"
                                % (what, _rank_label(args)), "data": "synthetic", "rows": rows}))


def run_parts(args):
    """Component timings on one GPU: the setup sweep alone, or the apply alone."""
    import torch
    import paper_1007_4290_gb300 as hs
    w = synth.workload(args.workload)
    n = w["n"]
    c_d = torch.tensor(w["c"], device="cuda")
    prec = hs.FP64 if args.fp64 else hs.MIXED
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = hs.hsweep_setup(c_d, w["omega"], w["pml"], w["eps_H"],
                        hs.default_opts(precision=prec, team=args.team, groups=args.groups, sweep_tc=args.sweep_tc,
                                        strong_rank=args.strong_rank))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    out = {"workload": args.workload, "n": n, "precision": "fp64" if args.fp64 else "mixed", "setup_s": setup_s,
           "strong_rank": args.strong_rank, "info": h.info()}
    if args.apply_only:
        nrhs = args.apply_only
        F = w["f"].reshape(w["f"].shape[0], -1)
        reps = (nrhs + F.shape[0] - 1) // F.shape[0]
        R = torch.tensor(np.concatenate([F] * reps)[:nrhs], device="cuda")
        Z = torch.empty_like(R)
        for _ in range(max(1, args.warmup)):
            h.apply(R, Z)
        h.profile(True)
        h.stats(reset=True)
        torch.cuda.synchronize()
        for _ in range(args.steps):
            h.apply(R, Z)
        torch.cuda.synchronize()
        launches, sweeps, sweep_ms = h.stats(reset=True)
        flops, bytes_, _ = sweep_work(h, n, nrhs, out["info"]["bytes_per_entry"])
        avg = sweep_ms / max(1, sweeps)
        out.update({"nrhs": nrhs, "apply_ms": avg, "plan": h.sweep_plan(nrhs),
                    "tflops": flops / (avg / 1e3) / 1e12, "hbm_gbs": bytes_ / (avg / 1e3) / 1e9})
    h.free()
    print(json.dumps(out))


def run_reference(args, world, rank):
    """The oracle arm: each step is a bounded sample of the same workload on the host
    cores (the oracle as it stands), on rank 0 only."""
    if rank != 0:
        return
    vals = []
    t0 = time.perf_counter()
    budget = max(5.0, 20.0 / max(1, args.steps + args.warmup) * 3)
    for k in range(args.warmup + args.steps):
        r = run_cpu_sample_subprocess(budget, 4.0)
        if k >= args.warmup:
            vals.append(r)
    elapsed = time.perf_counter() - t0
    value = float(np.median([v["value"] for v in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "oracle complex128"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": vals[-1]["sample"] + " (4 applies per solve assumed)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": elapsed}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
