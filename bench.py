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

if "--cpu-single" in sys.argv:
    # one BLAS thread for the single-thread oracle timings (read when numpy loads BLAS)
    for _k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_k] = "1"

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


def strong_sweep_work(n, R, nrhs, elem_bytes):
    """The same for the sweep on the strongly admissible format (sweep_strong.cu): per layer
    step and row, its near-field entries (its leaf and the neighbouring leaves) once and
    the R entries of every block of its clusters' interaction lists twice (reduction and
    expansion) per RHS; the records, stored entries included, are read once per step."""
    L, sz = _tree_sizes(n)
    nleaves = 1 << L
    near = far = stored = 0
    for j in range(nleaves):
        lam = nleaves + j
        s = sz[lam]
        sl = sz[lam - 1] if j > 0 else 0
        sr = sz[lam + 1] if j < nleaves - 1 else 0
        near += s * (s + sl + sr)
        stored += (s * ((s + sl + sr + 3 * R * (L - 1)) | 1) + 1) // 2 * 2
        for d in range(2, L + 1):
            c = lam >> (L - d)
            cl = c - (1 << d)
            offs = (-3, -2, 2) if cl & 1 else (-2, 2, 3)
            far += s * R * sum(1 for o in offs if 0 <= cl + o < (1 << d))
    steps = 2 * n - 1
    flops = 8.0 * nrhs * steps * (near + 2 * far)
    fac_bytes = steps * stored * elem_bytes
    vec_bytes = nrhs * n * n * (16 + 16 + 2 * elem_bytes)
    return flops, fac_bytes + vec_bytes, n * stored


# DRAM bytes (read + write) of one sweep launch, from ncu captures summarised in profiles/,
# keyed by workload and right-hand sides, with the SHA-256 of the kernel's device code they
# were taken on (kernel_source_digest): a changed kernel reports null instead of a stale
# number.
SWEEP_TRAFFIC = {
    # profiles/sweep_team_n1023_random_64rhs_dram.md: 3.979 GB read + 1.570 GB written
    "n1023_random/64": {"sha256": "ff634412e7829a3112e9c3af7488f956594a665fdbb4c8ba0cffe8587762d675",
                        "bytes": 5.5496e9},
}
TEAM_KERNEL_SRC = os.path.join(ROOT, "paper_1007_4290_gb300", "csrc", "sweep_team.cu")
STRONG_KERNEL_SRC = os.path.join(ROOT, "paper_1007_4290_gb300", "csrc", "sweep_strong.cu")
# the same for the sweep on the strongly admissible format (R = 2)
STRONG_TRAFFIC = {
    # profiles/sweep_strong_n1023_random_64rhs_dram.md: 2.631 GB read + 1.570 GB written
    "n1023_random/64": {"sha256": "4ff4aa8c37988400c0b7d1c986c746426f79883dc526ae5b5aaf1261827af431", "bytes": 4.2015e9},
}


def recorded_strong_traffic(workload, nrhs):
    rec = STRONG_TRAFFIC.get("%s/%d" % (workload, nrhs))
    if rec is None or not os.path.exists(STRONG_KERNEL_SRC):
        return None
    digest = kernel_source_digest(STRONG_KERNEL_SRC, b"struct StrongPack {")
    return rec["bytes"] if digest == rec["sha256"] else None


def kernel_source_digest(path=None, marker=b"struct TeamConfig {"):
    """SHA-256 of a sweep kernel's device code: its source up to the host-side part (the
    line `marker`) and the shared device helpers it includes (sweep_common.cuh)."""
    import hashlib
    path = path or TEAM_KERNEL_SRC
    h = hashlib.sha256()
    with open(path, "rb") as fh:
        src = fh.read()
    cut = src.find(marker)
    h.update(src[:cut] if cut > 0 else src)
    common = os.path.join(os.path.dirname(TEAM_KERNEL_SRC), "sweep_common.cuh")
    if os.path.exists(common):
        with open(common, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(workload, nrhs):
    rec = SWEEP_TRAFFIC.get("%s/%d" % (workload, nrhs))
    if rec is None or not os.path.exists(TEAM_KERNEL_SRC):
        return None
    return rec["bytes"] if kernel_source_digest() == rec["sha256"] else None


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
# CPU baseline: the oracle as it stands (Algorithms 2.5/2.6 in complex128 NumPy, and the
# sparse direct solve), on the host cores of the GPU machine.
def host_info():
    """Logical CPUs and the CPU model name of this host."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine()}


def oracle_chain(w, stop, log=None):
    """Algorithm 2.5 of the oracle (weak H-matrices, eps_H, rank cap 48) from layer 0
    until every layer is built or stop() is true.  Returns the T~_m built, the wall time
    of each layer and its stored entries (symmetric count: one factor pair per block)."""
    from oracle.assemble import Discretization
    from oracle.hmatrix import Trunc, hinv, hsub, tree_depth
    from oracle.sweep_h import tridiag_H
    disc = Discretization(w["c"], w["omega"], w["pml"])
    n = disc.n
    tr = Trunc(w["eps_H"], 48)
    L = tree_depth(n, 8)
    T, sec, ent = [], [], []
    for m in range(n):
        if m >= 2 and stop():
            break
        t0 = time.perf_counter()
        Amm = tridiag_H(disc.diag[m], disc.east[m, 1:-1], 0, 0, L)
        S = Amm if m == 0 else hsub(Amm, T[m - 1].diagmul(dl=disc.A_off(m), dr=disc.A_off(m)), tr)
        T.append(hinv(S, tr))
        sec.append(time.perf_counter() - t0)
        ent.append(sum(U.size for _, _, _, U, _ in T[m].blocks()))
        if log and m % 100 == 0:
            log("layer %d: %.1f s" % (m, sum(sec)))
    return disc, T, sec, ent


def oracle_apply_steps(disc, T, f):
    """The forward and backward sweeps of Algorithm 2.6 over the layers in T (all of
    them when T is complete); returns (seconds per layer step, z or None)."""
    n, ms = disc.n, len(T)
    u = f.reshape(n, n)[:ms].copy()
    w = [None] * ms
    t0 = time.perf_counter()
    for k in range(ms):
        w[k] = T[k].matvec(u[k])
        if k + 1 < ms:
            u[k + 1] = u[k + 1] - disc.A_off(k + 1) * w[k]
    u[ms - 1] = w[ms - 1]
    for k in range(ms - 2, -1, -1):
        u[k] = w[k] - T[k].matvec(disc.A_off(k + 1) * u[k + 1])
    dt = time.perf_counter() - t0
    return dt / (2 * ms - 1)


def cpu_baseline_run(out_json, uref_npy, stop_file, hard_s):
    """The CPU leg of the bench, run in its own process while the GPU legs run (started
    before any GPU call).  (1) O4: the oracle's setup chain from layer 0 over the whole
    domain, or until hard_s seconds (or stop_file appears), every layer timed; then its sweeps over
    all built layers, and, when the chain is complete, one whole preconditioned GMRES solve
    of source 0 (oracle.gmres, tolerance SOLVE_TOL).  (2) O2: the sparse direct solve of
    source 0 (factor and solve timed), whose solution is saved for the error of the GPU
    solutions.  Writes raw measurements; bench.py composes the baseline from them."""
    import numpy as np
    from oracle.direct import SparseLU
    from oracle.gmres import preconditioned_solve
    from oracle.sweep_h import HSweep
    w = synth.workload(WORKLOAD)
    t_start = time.perf_counter()
    stop = lambda: os.path.exists(stop_file) or time.perf_counter() - t_start > hard_s
    res = dict(host_info(), blas_threads=int(os.environ.get("OMP_NUM_THREADS", "0") or 0))
    disc, T, sec, ent = oracle_chain(w, stop)
    n = disc.n
    f0 = w["f"][0].ravel().astype(complex)
    res.update(layers_built=len(T), n=n, setup_layer_s=sec, layer_entries=ent)
    res["apply_step_s"] = oracle_apply_steps(disc, T, f0)
    if len(T) == n:
        H = HSweep.__new__(HSweep)
        H.disc, H.T = disc, T
        A = disc.matrix()
        t0 = time.perf_counter()
        _, it, _ = preconditioned_solve(A, H.apply, f0, SOLVE_TOL)
        res.update(solve_s=time.perf_counter() - t0, gmres_iters=it)
    del T
    t0 = time.perf_counter()
    lu = SparseLU(disc)
    t1 = time.perf_counter()
    u_ref = lu.solve(f0)
    res.update(o2_factor_s=t1 - t0, o2_solve_s=time.perf_counter() - t1)
    np.save(uref_npy, u_ref)
    with open(out_json, "w") as fh:
        json.dump(res, fh)


def run_cpu_single(names):
    """The oracle on one host thread (BLAS threads = 1) for the small configurations: the
    setup chain of Algorithm 2.5 over every layer, the sweeps of Algorithm 2.6, one whole
    preconditioned GMRES solve of source 0 at the workload's tolerance, and the sparse
    direct solve (O2).  One JSON line per workload; no GPU is used."""
    from oracle.direct import SparseLU
    from oracle.gmres import preconditioned_solve
    from oracle.sweep_h import HSweep
    info = host_info()
    for name in names:
        w = synth.workload(name)
        t0 = time.perf_counter()
        disc, T, sec, ent = oracle_chain(w, lambda: False)
        setup_s = time.perf_counter() - t0
        f0 = w["f"][0].ravel().astype(complex)
        step_s = oracle_apply_steps(disc, T, f0)
        H = HSweep.__new__(HSweep)
        H.disc, H.T = disc, T
        A = disc.matrix()
        t0 = time.perf_counter()
        u, it, _ = preconditioned_solve(A, H.apply, f0, w["tol"])
        solve_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        lu = SparseLU(disc)
        t1 = time.perf_counter()
        u_ref = lu.solve(f0)
        t2 = time.perf_counter()
        err = float(np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref))
        print(json.dumps({"cpu_single": name, "n": disc.n, "threads": 1, "eps_H": w["eps_H"], "tol": w["tol"],
                          "o4_setup_s": setup_s, "o4_apply_ms": 1e3 * step_s * (2 * disc.n - 1),
                          "o4_solve_s": solve_s, "gmres_iters": it, "rel_err_vs_direct": err,
                          "o2_factor_s": t1 - t0, "o2_solve_s": t2 - t1,
                          "nproc": info["nproc"], "cpu_model": info["cpu_model"]}), flush=True)


def start_cpu_baseline(tmpdir, hard_s=600.0):
    """Launch cpu_baseline_run in a new process with BLAS threads = all host cores but two
    (left to the GPU legs' host threads and the clock sampler)."""
    threads = max(1, (os.cpu_count() or 2) - 2)
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads))
    paths = {k: os.path.join(tmpdir, k) for k in ("cpu.json", "uref.npy", "stop")}
    proc = subprocess.Popen([sys.executable, os.path.abspath(__file__), "--cpu-baseline-run", paths["cpu.json"],
                             paths["uref.npy"], paths["stop"], str(hard_s)], env=env,
                            stdout=subprocess.DEVNULL, stderr=subprocess.PIPE, text=True)
    return proc, paths, threads


def finish_cpu_baseline(proc, paths, threads, applies_per_solve, timeout_s=900.0):
    """Wait for the CPU process (its chain stops by itself at its time limit) and compose
    the baseline: measured when the chain was complete (one whole solve), else the built
    layers' measured setup time plus the last tenth's mean per-layer time for the rest, and
    the measured per-step apply time x (2n - 1) steps x applies_per_solve."""
    import numpy as np
    try:
        _, err = proc.communicate(timeout=timeout_s)
    except subprocess.TimeoutExpired:
        proc.kill()
        return {"error": "cpu baseline process did not finish in %.0f s" % timeout_s}, None
    if proc.returncode != 0 or not os.path.exists(paths["cpu.json"]):
        return {"error": "cpu baseline failed: " + (err or "")[-300:]}, None
    with open(paths["cpu.json"]) as fh:
        r = json.load(fh)
    u_ref = np.load(paths["uref.npy"])
    n, built = r["n"], r["layers_built"]
    sec = r["setup_layer_s"]
    complete = built == n
    if complete:
        setup_s = sum(sec)
        solve_s = r["solve_s"]
        how = ("oracle H-sweep (Algorithms 2.5/2.6, weak, eps_H 1e-6, rank cap 48) at the full workload: "
               "setup of all %d layers %.1f s, one whole GMRES solve of source 0 %.2f s (%d steps); nothing "
               "extrapolated" % (n, setup_s, solve_s, r["gmres_iters"]))
    else:
        tail = sec[-max(1, built // 10):]
        setup_s = sum(sec) + (n - built) * float(np.mean(tail))
        solve_s = applies_per_solve * r["apply_step_s"] * (2 * n - 1)
        how = ("oracle H-sweep (Algorithms 2.5/2.6, weak, eps_H 1e-6, rank cap 48): setup chain from layer 0 "
               "through %d of %d layers in %.1f s while the GPU legs ran (the remaining layers at the mean "
               "time of the last tenth built: ranks still grow there, so the CPU estimate is optimistic); "
               "sweeps over the built layers %.2f ms per layer step; per-solve time = %.0f applies x %d layer "
               "steps (extrapolated)" % (built, n, sum(sec), 1e3 * r["apply_step_s"], applies_per_solve,
                                         2 * n - 1))
    out = {"value": 1.0 / solve_s, "unit": "solves/s", "cores": threads, "kind": "oracle", "sample": how,
           "nproc": r["nproc"], "cpu_model": r["cpu_model"], "blas_threads": r["blas_threads"],
           "setup_s": setup_s, "setup_measured": complete, "layers_built": built,
           "o2_direct": {"factor_s": r["o2_factor_s"], "solve_s": r["o2_solve_s"], "cores": 1,
                         "what": "oracle sparse LU (SuperLU) of A at n = %d, then one solve" % n}}
    if complete:
        out["gmres_iters_oracle"] = r["gmres_iters"]
    return out, u_ref


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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64", action="store_true",
                    help="with --apply-only / --setup-only: FP64 factors instead of mixed precision")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the plain FP64 comparator of the default run (its setup takes minutes)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline of the default run")
    ap.add_argument("--no-strong", action="store_true",
                    help="skip the strongly admissible sweep (R = 2) of the default run")
    ap.add_argument("--cpu-seconds", type=float, default=600.0,
                    help="longest time the CPU baseline's setup chain may run beside the GPU legs")
    ap.add_argument("--krylov-lowp", type=int, default=0,
                    help="inner GMRES of the mixed solve in FP32 arithmetic (off by default)")
    ap.add_argument("--cpu-baseline-run", nargs=4, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-single", default="",
                    help="comma-separated workloads (n64_const,n511_lens): the oracle on one host thread "
                         "(setup, apply, one solve, the direct solve), one JSON line each; no GPU")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="synthetic workload (n1023_random, n511_lens, n64_const, n2047_random)")
    ap.add_argument("--apply-only", type=int, default=0, metavar="NRHS",
                    help="time only the sweep apply (Algorithm 2.6) on NRHS right-hand sides")
    ap.add_argument("--setup-only", action="store_true", help="time only the setup sweep (Algorithm 2.5)")
    ap.add_argument("--team", type=int, default=0, help="with --apply-only: CTAs per sweep team (0 = automatic)")
    ap.add_argument("--groups", type=int, default=0, help="with --apply-only: right-hand sides per team (0 = automatic)")
    ap.add_argument("--core-kernel", type=int, default=0,
                    help="with --setup-only / --apply-only: recompression cores on the autotuned kernel (0), "
                         "CUDA cores (1) or tensor cores (2)")
    ap.add_argument("--team-threads", type=int, default=0,
                    help="with --apply-only: threads per CTA of the team sweep (512, 256; 0 = automatic)")
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

    if args.cpu_baseline_run is not None:
        a = args.cpu_baseline_run
        cpu_baseline_run(a[0], a[1], a[2], float(a[3]))
        return
    if args.cpu_single:
        run_cpu_single([x for x in args.cpu_single.split(",") if x])
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

    # the CPU baseline runs in its own process beside the GPU legs; it starts before the
    # first GPU call (rank 0 of a one-process run only)
    cpu_job = None
    if rank == 0 and world == 1 and not args.no_cpu and args.workload == WORKLOAD:
        import tempfile
        cpu_tmp = tempfile.mkdtemp(prefix="hsweep_cpu_")
        cpu_job = start_cpu_baseline(cpu_tmp, args.cpu_seconds)

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
    h = hs.hsweep_setup(c_d, omega, pml, eps, hs.default_opts(precision=hs.MIXED, krylov_lowp=args.krylov_lowp))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    info = h.info()
    setup_tuning = h.setup_tuning()
    # ranks of the factorised blocks per depth (min / mean / max over every 16th layer)
    Ld, _ = _tree_sizes(n)
    per_depth = {d: [] for d in range(1, Ld + 1)}
    for m in range(0, n, 16):
        rk = h.layer_ranks(m)
        for v in range(2, 1 << (Ld + 1)):
            per_depth[v.bit_length() - 1].append(rk[v])
    ranks = {str(d): [int(min(r)), round(float(np.mean(r)), 1), int(max(r))] for d, r in per_depth.items() if r}

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
    roof["kernel"] = {2: "sweep_team_kernel"}.get(plan["tma"], "sweep_kernel") + "<c64>"
    roof["plan"] = plan
    roof["launch_ms"] = avg_s * 1e3
    roof["hbm_gbs_achieved"] = bytes_ / avg_s / 1e9
    roof["hbm_frac"] = roof["hbm_gbs_achieved"] / peaks["hbm_gbs"]
    roof["algorithmic_flops_per_launch"] = flops
    roof["algorithmic_bytes_per_launch"] = bytes_

    # the apply alone at 1 and 16 right-hand sides (the HBM-bound end of the sweep): CUDA
    # events around each launch, achieved bandwidth of the algorithmic bytes
    apply_hbm = {}
    for nr in (1, 16):
        Rn = f_d[:nr].clone()
        Zn = torch.empty_like(Rn)
        for _ in range(3):
            h.apply(Rn, Zn)
        h.stats(reset=True)
        h.profile(True)
        for _ in range(10):
            h.apply(Rn, Zn)
        h.profile(False)
        _, sw_n, swms_n = h.stats(reset=True)
        fl_n, by_n, _ = sweep_work(h, n, nr, info["bytes_per_entry"])
        t_n = swms_n / max(1, sw_n) / 1e3
        pk, _ = _peaks()
        apply_hbm[str(nr)] = {"launch_ms": t_n * 1e3, "algorithmic_bytes": by_n, "gbs": by_n / t_n / 1e9,
                              "hbm_frac": by_n / t_n / 1e9 / pk["hbm_gbs"], "tflops": fl_n / t_n / 1e12,
                              "us_per_layer_step": t_n * 1e6 / (2 * n - 1)}
        del Rn, Zn

    # the batched apply of all the sources as one graph-captured launch: the handle moves to
    # a stream that can be captured, h.apply is captured once (the exchange memset and the
    # cooperative sweep kernel) and the graph replayed; CUDA events around the replays
    gstream = torch.cuda.Stream(device=dev)
    gstream.wait_stream(stream)
    h.set_stream(gstream)
    try:
        Zg = torch.empty_like(f_d)
        with torch.cuda.stream(gstream):
            h.apply(f_d, Zg)             # the handle's buffers sized outside the capture
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gstream):
            h.apply(f_d, Zg)
        g_reps = 10
        ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(gstream):
            for _ in range(2):
                graph.replay()
            ga.record(gstream)
            for _ in range(g_reps):
                graph.replay()
            gb.record(gstream)
            Zref = h.apply(f_d)
        gstream.synchronize()
        apply_graph = {"nrhs": nrhs, "launch_ms": ga.elapsed_time(gb) / g_reps, "replays": g_reps,
                       "identical_to_eager": bool(torch.equal(Zg, Zref)),
                       "what": "hsweep_apply captured once into a CUDA graph on the handle's stream "
                               "(exchange memset + cooperative sweep kernel), replayed back to back"}
        del graph, Zg, Zref
    except Exception as e:          # reported in the line; the rest of the run goes on
        apply_graph = {"error": str(e)[:300]}
    gstream.synchronize()
    stream.wait_stream(gstream)
    h.set_stream(stream)

    # the mixed solution of source 0 (the last timed step's), for its error against the
    # direct solve of the CPU leg
    u_mixed0 = u_d[0].cpu().numpy() if rank == 0 else None

    # the plain FP64 comparator (Section 8(d) of the measurement plan): complex128 factors
    # and sweeps, the same team kernel, one right-hand side per call, its setup timed
    fp64 = None
    if not args.no_fp64:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h64 = hs.hsweep_setup(c_d, omega, pml, eps, hs.default_opts(precision=hs.FP64))
        torch.cuda.synchronize()
        s64 = time.perf_counter() - t0
        u1 = torch.zeros_like(f_d[:1])
        for _ in range(2):
            u1.zero_()
            h64.solve(f_d[:1], SOLVE_TOL, u=u1)
        k64 = min(8, nrhs)
        h64.stats(reset=True)
        h64.profile(True)
        torch.cuda.synchronize()
        e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e4.record(stream)
        its, rrs = [], []
        for s_ in range(k64):
            u1.zero_()
            _, it1, rr1 = h64.solve(f_d[s_:s_ + 1], SOLVE_TOL, u=u1)
            its.append(it1[0])
            rrs.append(rr1[0])
            if s_ == 0:
                u64_0 = u1[0].cpu().numpy()     # outside the events' span would need a sync anyway
        e5.record(stream)
        torch.cuda.synchronize()
        h64.profile(False)
        _, sw64, swms64 = h64.stats(reset=True)
        ms64 = e4.elapsed_time(e5)
        inf64 = h64.info()
        fp64 = {"solves_per_s": k64 / (ms64 / 1e3), "setup_s": s64, "nrhs_per_call": 1, "solves_timed": k64,
                "gmres_iters": its, "relres_max": max(rrs), "sweep_launches": sw64,
                "sweep_launch_ms": swms64 / max(1, sw64),
                "factor_gb": inf64["entries"] * inf64["bytes_per_entry"] / 1e9,
                "note": "the device->host copy of source 0's solution sits inside this span"}
        h64.free()

    # the sweep on the strongly admissible format (strong_rank = 2, the configuration of the
    # paper's experiments) on the same workload: its own setup, then the 64-RHS apply timed
    # with CUDA events around each launch
    strong = None
    if not args.no_strong:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hst = hs.hsweep_setup(c_d, omega, pml, eps, hs.default_opts(precision=hs.MIXED, strong_rank=2))
        torch.cuda.synchronize()
        s_st = time.perf_counter() - t0
        Zs = torch.empty_like(f_d)
        for _ in range(3):
            hst.apply(f_d, Zs)
        hst.stats(reset=True)
        hst.profile(True)
        for _ in range(10):
            hst.apply(f_d, Zs)
        hst.profile(False)
        _, sw_s, swms_s = hst.stats(reset=True)
        t_s = swms_s / max(1, sw_s) / 1e3
        fl_s, by_s, st_s = strong_sweep_work(n, 2, nrhs, info["bytes_per_entry"])
        strong = {"R": 2, "setup_s": s_st, "launch_ms": t_s * 1e3, "plan": hst.sweep_plan(nrhs),
                  "algorithmic_flops_per_launch": fl_s, "algorithmic_bytes_per_launch": by_s,
                  "traffic": recorded_strong_traffic(args.workload, nrhs),
                  "tflops": fl_s / t_s / 1e12, "gbs": by_s / t_s / 1e9, "stored_entries": st_s,
                  "what": "sweep_strong_kernel on the strongly admissible records (near field + rank-2 "
                          "interaction-list factors), 64 RHS, mixed precision"}
        hst.free()
        del Zs

    cpu, u_ref = None, None
    if cpu_job is not None:
        proc, paths, threads = cpu_job
        cpu, u_ref = finish_cpu_baseline(proc, paths, threads, applies_per_solve=(
            1 + float(np.mean(fp64["gmres_iters"])) if fp64 else 4.0))
    rel_err = None
    if u_ref is not None:
        nref = np.linalg.norm(u_ref)
        rel_err = {"source": 0, "mixed": float(np.linalg.norm(u_mixed0 - u_ref) / nref),
                   "reference": "oracle sparse LU (SuperLU) of A, complex128, on the host",
                   "targets": {"metric": 1e-6, "mixed": 1e-5, "fp64": 1e-6}}
        if fp64 is not None:
            rel_err["fp64"] = float(np.linalg.norm(u64_0 - u_ref) / nref)
    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("c64 H-factors, setup products and sweeps; f64 GMRES (Arnoldi, A-products, norms), "
                      "residuals, refinement and leaf inversions" if not args.krylov_lowp else
                      "c64 H-factors, setup products and sweeps; inner GMRES in f32 arithmetic on f64 vectors; "
                      "f64 residuals, refinement and leaf inversions"),
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "N": n * n, "omega_over_2pi": omega / (2 * np.pi),
                       "pml": pml, "eps_H": eps, "nrhs": nrhs, "precision": "mixed", "tol": SOLVE_TOL,
                       "parallelism": "replica per GPU, sources sharded" if world > 1 else "1 GPU",
                       "l2": "inputs larger than L2 (%.2f GB RHS batch, factors %.2f GB)" % (
                           nrhs * n * n * 16 / 1e9, stored * info["bytes_per_entry"] / 1e9)},
            "setup_s": setup_s,
            "setup_tuning": setup_tuning,
            "ranks_per_depth": ranks,
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
            "apply_only": apply_hbm,
            "apply_graph": apply_graph,
            "strong_sweep": strong,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        line["config"]["krylov"] = "fp32 inner arithmetic" if args.krylov_lowp else "fp64"
        if fp64 is not None:
            line["fp64"] = fp64
            line["mixed_over_fp64"] = value / fp64["solves_per_s"]
        if rel_err is not None:
            line["rel_err_vs_direct"] = rel_err
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
                                        strong_rank=args.strong_rank, team_threads=args.team_threads,
                                        core_kernel=args.core_kernel))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    out = {"workload": args.workload, "n": n, "precision": "fp64" if args.fp64 else "mixed", "setup_s": setup_s,
           "strong_rank": args.strong_rank, "info": h.info(), "setup_tuning": h.setup_tuning()}
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
        plan = h.sweep_plan(nrhs)
        if plan["tma"] == 3:
            flops, bytes_, _ = strong_sweep_work(n, args.strong_rank, nrhs, out["info"]["bytes_per_entry"])
        else:
            flops, bytes_, _ = sweep_work(h, n, nrhs, out["info"]["bytes_per_entry"])
        avg = sweep_ms / max(1, sweeps)
        out.update({"nrhs": nrhs, "apply_ms": avg, "plan": plan, "algorithmic_flops": flops,
                    "algorithmic_bytes": bytes_,
                    "tflops": flops / (avg / 1e3) / 1e12, "hbm_gbs": bytes_ / (avg / 1e3) / 1e9})
    h.free()
    print(json.dumps(out))


# applies of M per solve of the GPU arm's mixed solve at this workload (bench.py's
# sweep_launches_per_step: M f, two inner GMRES steps, the residual check of the one FP64
# refinement step and its inner GMRES step); the reference arm's per-solve time uses the
# same count
REFERENCE_APPLIES_PER_SOLVE = 5


def run_reference(args, world, rank):
    """The oracle arm: each step is a bounded sample of the same workload on the host
    cores (the oracle as it stands, BLAS threads = all cores), on rank 0 only: the setup
    chain of Algorithm 2.5 from layer 0 for a few seconds, then the sweeps of Algorithm 2.6
    over the layers built.  The per-solve time is extrapolated: the measured time per
    layer step x (2n - 1) steps x REFERENCE_APPLIES_PER_SOLVE."""
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, str(threads))
    w = synth.workload(WORKLOAD)
    n = w["n"]
    f0 = w["f"][0].ravel().astype(complex)
    budget = max(2.0, min(6.0, 150.0 / max(1, args.steps + args.warmup)))
    per, walls, built = [], [], []
    t_all = time.perf_counter()
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        disc, T, sec, _ = oracle_chain(w, lambda: time.perf_counter() - t0 > budget)
        step_s = oracle_apply_steps(disc, T, f0)
        if k >= args.warmup:
            per.append(step_s)
            walls.append(time.perf_counter() - t0)
            built.append(len(T))
    elapsed = time.perf_counter() - t_all
    step_s = float(np.median(per))
    solve_s = REFERENCE_APPLIES_PER_SOLVE * step_s * (2 * n - 1)
    value = 1.0 / solve_s
    info = host_info()
    sample = ("oracle H-sweep (Algorithms 2.5/2.6, weak, eps_H 1e-6, rank cap 48), each step a bounded sample: "
              "the setup chain from layer 0 for %.0f s (%d of %d layers built, the absorbing layers and the first "
              "interior ones, where ranks are lowest: optimistic for the CPU), then the sweeps over those layers, "
              "%.2f ms per layer step (median of %d steps); per-solve time extrapolated = %d applies x %d layer "
              "steps = %.1f s" % (budget, int(np.median(built)), n, 1e3 * step_s, len(per),
                                  REFERENCE_APPLIES_PER_SOLVE, 2 * n - 1, solve_s))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(walls)),
            "ms_per_step_is": "wall time of one bounded sample step (the per-solve time is extrapolated)",
            "extrapolated": True, "solve_s_extrapolated": solve_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "oracle complex128"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle",
                             "sample": sample, "nproc": info["nproc"], "cpu_model": info["cpu_model"]},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": elapsed}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
