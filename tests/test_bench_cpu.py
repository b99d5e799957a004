"""bench.py's single-thread oracle timings (the CPU reference figures of the small
configurations): one JSON line per workload with the oracle's setup, apply, solve and
direct-solve times, run on the host alone."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_cpu_single_line_for_the_smallest_workload():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-single", "n64_const"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [json.loads(x) for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["cpu_single"] == "n64_const" and d["n"] == 64 and d["threads"] == 1
    assert d["o4_setup_s"] > 0 and d["o4_solve_s"] > 0 and d["o2_factor_s"] > 0
    # eps_H = 1e-9 and tol = 1e-8: the oracle's preconditioned solve reaches the direct solution
    assert d["gmres_iters"] <= 3
    assert d["rel_err_vs_direct"] < 1e-7


def test_traffic_keys_follow_the_device_code_only(tmp_path):
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    # the committed DRAM captures belong to the committed kernels: the bench line carries them
    assert bench.recorded_traffic("n1023_random", 64) is not None
    assert bench.recorded_strong_traffic("n1023_random", 64) is not None
    # an edit of the host part (after the marker) keeps the key, an edit of the device part drops it
    src = open(bench.TEAM_KERNEL_SRC, "rb").read()
    cut = src.find(b"struct TeamConfig {")
    assert cut > 0
    p_host = tmp_path / "host_edit.cu"
    p_host.write_bytes(src + b"\n// host-side edit\n")
    p_dev = tmp_path / "device_edit.cu"
    p_dev.write_bytes(src[:cut] + b"// device-side edit\n" + src[cut:])
    d0 = bench.kernel_source_digest()
    assert bench.kernel_source_digest(str(p_host)) == d0
    assert bench.kernel_source_digest(str(p_dev)) != d0


def _bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod2", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_strong_sweep_work_counts_the_near_field_and_the_interaction_lists():
    """The algorithmic flops of the strong-format sweep's roofline: per layer step and row,
    the dense near field (its leaf and the two neighbouring leaves) once and the R columns of
    every block of its clusters' interaction lists (Section 2.3; the oracle's Clusters) twice
    per right-hand side, over 2n - 1 steps."""
    from oracle.hmatrix_strong import Clusters
    bench = _bench()
    for n, R, nrhs in [(31, 2, 1), (127, 2, 3), (255, 1, 2), (100, 3, 1), (1023, 2, 64)]:
        flops, _, _ = bench.strong_sweep_work(n, R, nrhs, 8)
        ct = Clusters(n, 8)
        L, nl = ct.L, 1 << ct.L
        near = far = 0
        for i in range(nl):
            s = ct.size(L, i)
            near += s * sum(ct.size(L, j) for j in (i - 1, i, i + 1) if 0 <= j < nl)
            for lev in range(1, L + 1):
                far += s * R * len(ct.interaction_list(lev, i >> (L - lev)))
        assert flops == 8.0 * nrhs * (2 * n - 1) * (near + 2 * far), (n, R)


def test_weak_sweep_work_counts_the_entries_of_the_oracle_layers():
    """The algorithmic flops of the sibling-pair sweep's roofline, from a handle's rank table,
    against the H-matrices of the oracle's setup (Algorithm 2.5) on the same tree: per layer
    step the dense leaves once and both factors of every off-diagonal block (V^t x, then U q),
    8 real flops per complex multiply-add, forward over n layers and backward over n - 1."""
    from oracle.assemble import Discretization
    from oracle.sweep_h import HSweep
    import numpy as np
    import synth
    bench = _bench()
    n, nrhs = 63, 2
    disc = Discretization(synth.velocity_random(n, 1 / 8, 1), 2 * np.pi * 4, 6)
    H = HSweep(disc, 1e-6, rmax=12)
    L, sz = bench._tree_sizes(n)
    assert L == H.L
    # heap index of every node of the bisection tree by (depth, first row)
    node, lo = {}, {1: 0}
    for v in range(1, 1 << (L + 1)):
        d = v.bit_length() - 1
        if v > 1:
            p = v // 2
            lo[v] = lo[p] + (sz[2 * p] if v & 1 else 0)
        node[(d, lo[v])] = v

    class FakeHandle:
        def layer_ranks(self, m):
            rk = [0] * (1 << (L + 1))
            for d, (r0, _), _, U, _ in H.T[m].blocks():
                rk[node[(d, r0)]] = U.shape[1]
            return rk

    flops, _, _ = bench.sweep_work(FakeHandle(), n, nrhs, 8)
    macs = []
    for T in H.T:
        leaf = sum(t.hi - t.lo for t in T.leaves() for _ in range(t.hi - t.lo))
        lowrank = sum(U.size + V.size for _, _, _, U, V in T.blocks())
        macs.append(leaf + lowrank)
    expect = 8.0 * nrhs * (sum(macs) + sum(macs[:-1]))
    assert flops == expect
