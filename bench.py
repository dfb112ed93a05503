#!/usr/bin/env python
"""Benchmark of joint-cut HSF simulation on one GB300 (or N, one process per GPU).

Workload (default): n = 30 qubits split 15|15, 20 layers of Haar U(2) with CZ
brickwork inside each half, 8 jointly cut blocks of 4 RZZ (+ interleaved U(2)) on the
qubit pair (14, 15) -> 4^8 = 65536 paths (2^32 with per-gate cuts); amplitudes of 4096
seeded bitstrings, complex64 half states, FP64 cross-path sums.

A step is the whole hot path for one circuit: plan (validation, block products and
FP64 Schmidt SVD on the GPU, gate programs) + run (all paths' half-state sweeps and
the path sum) through the C ABI.  The metric is circuits per second.

Multi-GPU: each rank simulates its own circuit (seed + rank); there is no collective
on the data path ("scaling": "weak").

--impl reference times the FP64 CPU oracle on the host cores over a bounded sample
of paths of the same workload and reports the extrapolated circuits per second.
"""
from __future__ import annotations

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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HSF circuits/s (n=30 joint cut, 4096 bitstrings)"
UNIT = "circuits/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="c64", choices=["c64", "c128"])
    ap.add_argument("--no-extras", action="store_true", help="skip plain-cut and CPU baseline legs")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU-baseline sample time")
    ap.add_argument("--paths", type=int, default=0,
                    help="profiling aid: simulate only the first N paths (0 = all)")
    ap.add_argument("--budget-gb", type=float, default=0.0,
                    help="profiling aid: cap the workspace (path chunks shrink to fit)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5", "c1"],
                    help="c2 (default, n=30 bitstrings); c3: 64 uneven circuits in one CUDA graph "
                         "(window output, tensor-core path GEMM); c4: QAOA n=28 adjoint gradients; "
                         "c5: n=36, 2^20 bitstrings; c1: n=12 all amplitudes")
    ap.add_argument("--gemm", default="bf16x3", choices=["fp32", "bf16x3", "tf32x3", "tf32"])
    ap.add_argument("--tune", action="store_true", help="c3: autotune one circuit per qubit count")
    ap.add_argument("--max-n", type=int, default=0, help="c3 profiling aid: drop circuits above this n")
    ap.add_argument("--largest-only", action="store_true",
                    help="c3 profiling aid: run only the largest circuit once (no graph)")
    ap.add_argument("--leaf-dots", action="store_true",
                    help="c2 profiling aid: plan with HSF_FLAG_LEAF_DOTS (level 7 writes the leaf's dots)")
    return ap.parse_args()


def workload(rank: int = 0):
    from paper_2502_06959_gb300 import workloads as W
    return W.workload_c2(seed=2 + rank)


C2_CONFIG = {"workload": "n30_15x15_20layers_8blocks_4096bitstrings", "n": 30, "cut": 14, "paths": 4 ** 8,
             "bitstrings": 4096, "blocks": 8}
GOLDEN_C2 = os.path.join(ROOT, "tests", "golden", "c2_n30_amplitudes.json")
GOLDEN_C3 = os.path.join(ROOT, "tests", "golden", "c3_largest_window.json")


def load_golden(path):
    """Stored FP64 amplitudes written by a script under tests/golden/ from the oracle."""
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    rec["amps"] = np.array(rec["re"]) + 1j * np.array(rec["im"])
    return rec


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        # nvidia-smi is started, and its first sample awaited, before the caller's timed
        # region begins: its start-up would otherwise compete with the timed work
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        self.first = len(self.lines)       # samples from here on fall in the timed region
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines[getattr(self, "first", 0):] or self.lines[-1:]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM traffic per launch relative to the algorithmic bytes, from one ncu capture of the
# kernel (dram__bytes_read.sum + dram__bytes_write.sum over the launch's algorithmic
# bytes).  A ratio is valid only for the kernel it was taken on: the entry records the
# first 16 hex digits of the SHA-256 of that kernel's definition (from its __global__
# line to its closing brace) at capture time; host code and other kernels of the file
# may change without invalidating it.  The summaries named here hold the numbers and the
# commands.
PROFILED_TRAFFIC = {
    "sweep": {"ratio": 275.1 / 335.5, "source": "paper_2502_06959_gb300/csrc/sweep.cu",
              "kernel": "sweep_reg_kernel", "sha256": "1a9bade5309e94b9",
              "profile": "profiles/sweep_reg_level6_n30.md"},
    "level_f16": {"ratio": (268.8 + 878.2) / 1342.2, "source": "paper_2502_06959_gb300/csrc/gemm_tc.cu",
                  "kernel": "level_mma_f16_kernel", "sha256": "8185c06fa54cecd6",
                  "profile": "profiles/level_f16_level7_n30.md"},
    "leaf": {"ratio": (1883.1 + 7.0) / 2151.7, "source": "paper_2502_06959_gb300/csrc/accum.cu",
             "kernel": "leaf_contract_fact_kernel", "sha256": "f449d346010749b5",
             "profile": "profiles/leaf_contract_fact_n30.md"},
    # level 6 of the small n=30 case (levels 5 and 6 share the kernel; level 5's output
    # stayed in L2 there, so the larger launch's ratio stands for both)
    "level_mma": {"ratio": (67.7 + 207.6) / 335.5, "source": "paper_2502_06959_gb300/csrc/gemm_tc.cu",
                  "kernel": "level_mma_kernel", "sha256": "5846d163ab97848f",
                  "profile": "profiles/level_mma_levels56_n30.md"},
}


def _kernel_text(rel, kernel):
    """Source text of the __global__ function `kernel` in file `rel`."""
    with open(os.path.join(ROOT, rel)) as f:
        src = f.read()
    i = 0
    while True:
        i = src.find("__global__", i)
        if i < 0:
            return None
        j = src.find("{", i)
        head = src[i:j]
        if (" " + kernel + "(") in head or (" " + kernel + " (") in head:
            depth, k = 0, j
            while k < len(src):
                if src[k] == "{":
                    depth += 1
                elif src[k] == "}":
                    depth -= 1
                    if depth == 0:
                        return src[i:k + 1]
                k += 1
            return None
        i = j


def _kernel_hash(rel, kernel):
    import hashlib
    t = _kernel_text(rel, kernel)
    return hashlib.sha256(t.encode()).hexdigest()[:16] if t is not None else None


def traffic_per_launch(kind, algorithmic_bytes_per_launch):
    """ncu-derived DRAM bytes per launch, or None when no capture matches the kernel."""
    e = PROFILED_TRAFFIC.get(kind)
    if not e or _kernel_hash(e["source"], e["kernel"]) != e["sha256"]:
        return None
    return e["ratio"] * algorithmic_bytes_per_launch


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 1900.0, 2070.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle leg (the only place bench.py runs oracle/)
# ---------------------------------------------------------------------------
def _oracle_slice(args):
    n, gates, cut, blocks, bits, a, b = args
    import oracle.hsf_oracle as O
    out, _ = O.hsf_amplitudes(n, gates, cut, blocks, bitstrings=bits, path_range=(a, b))
    return out


def oracle_sample(pr, paths_per_core: int, cores: int, start: int = 0):
    """Oracle path sum over [start, start + cores*paths_per_core) on `cores` spawned
    processes; returns (amplitudes, seconds, paths)."""
    import multiprocessing as mp
    total = cores * paths_per_core
    jobs = [(pr.n, pr.gates, pr.cut, pr.blocks, pr.bitstrings, start + i * paths_per_core,
             start + (i + 1) * paths_per_core) for i in range(cores)]
    ctx = mp.get_context("spawn")
    # one BLAS thread per worker (inherited by the spawned processes): `cores` processes
    # use `cores` threads
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_slice, jobs[:1])            # start-up outside the timing
        t0 = time.perf_counter()
        parts = pool.map(_oracle_slice, jobs)
        dt = time.perf_counter() - t0
    return np.sum(parts, axis=0), dt, total


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def calibrate_paths_per_core(pr, target_s: float, cores: int):
    _, dt, tot = oracle_sample(pr, 1, cores)
    per_path_core = dt                        # seconds for one path on each core
    return max(1, int(target_s / max(per_path_core, 1e-3)))


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pr = workload(0)
    cores = cpu_cores()
    from paper_2502_06959_gb300.workloads import Problem  # noqa: F401  (inputs only)
    P = 4 ** 8
    per_step_target = max(2.0, 120.0 / max(1, args.steps + args.warmup))
    ppc = calibrate_paths_per_core(pr, per_step_target, cores)
    times, step_s = [], []
    for i in range(args.warmup + args.steps):
        _, dt, tot = oracle_sample(pr, ppc, cores, start=(i * cores * ppc) % P)
        if i >= args.warmup:
            times.append(dt / tot)          # seconds per path
            step_s.append(dt)
    sec_per_path = statistics.mean(times)
    value = 1.0 / (sec_per_path * P)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        # a step is a bounded sample of the circuit's paths: ms_per_step is its measured
        # wall time; value is extrapolated from it to all paths
        "ms_per_step": statistics.mean(step_s) * 1e3,
        "extrapolated": {"seconds_per_circuit": sec_per_path * P, "from_paths_per_step": ppc * cores},
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic",
        "config": dict(C2_CONFIG, sample_paths_per_step=ppc * cores),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{ppc * cores} of {P} paths per step, extrapolated"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def _timed(torch, stream, fn, steps):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _tuned_summary(tuned):
    """How often each tuned choice was taken over the circuits."""
    out = {}
    for v in tuned.values():
        key = f"tile{v['tile_bits']}/flags{v['flags']}/{v['gemm']}/budget={v['budget'] or 'full'}"
        out[key] = out.get(key, 0) + 1
    return out


def bench_other(args):
    """Secondary workloads (one GPU): c3 batched graph, c4 gradients, c5 n=36, c1 parity."""
    import torch
    from paper_2502_06959_gb300 import hsf
    from paper_2502_06959_gb300 import workloads as W
    torch.cuda.set_device(0)
    hsf.load_library()
    stream = torch.cuda.current_stream()
    hbm_peak, bf16_peak, sm_max, peak_src = peaks()
    line = {"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "data": "synthetic"}
    if args.workload == "c3":
        probs = W.workload_c3()
        if args.max_n:
            probs = [pr for pr in probs if pr.n <= args.max_n]
        if args.largest_only:
            pr = max(probs, key=lambda q: (q.n, len(q.blocks)))
            plan = hsf.Plan.from_problem(pr, precision="c64", gemm=args.gemm)
            window = min(1 << pr.n, 1 << 24)
            out = plan.run(window=window, check=True)
            torch.cuda.synchronize()
            print(json.dumps({"largest": pr.name, "paths": int(plan.info["num_paths"]), "window": window}))
            plan.close()
            return
        tuned = {}
        if args.tune:
            # one tuning per circuit shape (the cache key is the circuit's structure: the
            # same qubit count with another block count is another shape, and the best
            # path-GEMM form depends on the path count)
            import tempfile
            cache = os.path.join(tempfile.gettempdir(), "hsf_tune_cache.txt")
            for pr in probs:
                window = min(1 << pr.n, 1 << 24)
                tuned[pr.name] = hsf.hsf_tune(pr.n, pr.gates, pr.cut, pr.blocks, window=window, cache_path=cache,
                                              gemm=args.gemm)
        items = []
        for pr in probs:
            window = min(1 << pr.n, 1 << 24)
            opts = dict(tuned.get(pr.name, {}))
            opts.pop("budget", None)             # the batch shares one workspace
            gemm = opts.pop("gemm", args.gemm)
            plan = hsf.Plan.from_problem(pr, precision="c64", gemm=gemm, **opts)
            items.append(dict(plan=plan, window=window,
                              out=torch.empty(window, dtype=torch.complex128, device="cuda")))
        gstream = torch.cuda.Stream()          # graphs are recorded on a non-default stream
        batch = hsf.Batch(items, stream=gstream)
        for _ in range(args.warmup):
            batch.launch(gstream)
        l0 = hsf.hsf_launch_count()
        with ClockSampler(0) as clk:
            ms = _timed(torch, gstream, lambda: batch.launch(gstream), args.steps)
        launches = hsf.hsf_launch_count() - l0
        # the path GEMM of the largest circuit, timed alone with per-kernel events
        big = max(items, key=lambda it: it["plan"].n * 10 ** 6 + it["plan"].info["num_paths"])
        hsf.hsf_set_profiling(True)
        big["plan"].run(window=big["window"], out=big["out"])
        torch.cuda.synchronize()
        st = hsf.hsf_profile_collect(big["plan"].handle)
        hsf.hsf_set_profiling(False)
        w = st["window"]
        tf = w["flops"] / (w["ms"] / 1e3) / 1e12 if w["ms"] else 0.0
        paths = [it["plan"].info["num_paths"] for it in items]
        ns = [it["plan"].n for it in items]
        line.update({
            "metric": "HSF circuits/s (64 uneven circuits, one CUDA graph, window output)",
            "value": len(items) * args.steps / (ms / 1e3), "unit": "circuits/s",
            "ms_per_step": ms / args.steps, "dtype": "c64+" + args.gemm,
            "config": {"workload": "c3_64_uneven_n20to32_window2^24", "circuits": len(items),
                       "n_range": [min(ns), max(ns)], "paths_range": [min(paths), max(paths)],
                       "graph_kernel_nodes": batch.nodes, "tuned": bool(args.tune),
                       "tuned_choices": _tuned_summary(tuned),
                       "step": "one graph replay of hsf_run for all 64 plans"},
            "gpu_launches": int(launches),
            "roofline": {"bound": "tensor", "kernel": "path_gemm (largest circuit)", "achieved": tf,
                         "peak": bf16_peak, "unit": "TFLOP/s", "frac": tf / bf16_peak, "traffic": None,
                         "peak_source": peak_src + " (bf16 dense; counted flops = 3 bf16 products)",
                         "gemm_ms": w["ms"], "circuit_n": big["plan"].n,
                         "circuit_paths": big["plan"].info["num_paths"]},
            "clocks": clk.summary(),
        })
        batch.close()
        for it in items:
            it["plan"].close()
    elif args.workload == "c4":
        pr = W.workload_c4()
        bits = torch.from_numpy(pr.bitstrings.view(np.int64)).cuda()
        theta = torch.tensor(pr.params, dtype=torch.float64, requires_grad=True)

        def step():
            amps = hsf.HSFAmplitudes.apply(theta, pr, bits, "c64")
            loss = (amps.abs() ** 2).sum()
            theta.grad = None
            loss.backward()
        for _ in range(args.warmup):
            step()
        l0 = hsf.hsf_launch_count()
        with ClockSampler(0) as clk:
            ms = _timed(torch, stream, step, args.steps)
        launches = hsf.hsf_launch_count() - l0
        line.update({
            "metric": "QAOA gradients/s (n=28, p=4, 1024 bitstrings, adjoint through every path)",
            "value": args.steps / (ms / 1e3), "unit": "gradients/s", "ms_per_step": ms / args.steps,
            "dtype": "c64", "config": {"workload": "c4_qaoa_n28_p4_1024bitstrings", "params": int(pr.num_params),
                                       "step": "plan + forward + hsf_grad (autograd Function)"},
            "gpu_launches": int(launches), "clocks": clk.summary()})
    else:
        pr = W.workload_c5() if args.workload == "c5" else W.workload_c1()
        plan = hsf.Plan.from_problem(pr, precision="c64" if args.workload == "c5" else "c128")
        bits = None
        if pr.bitstrings is not None:
            bits = torch.from_numpy(pr.bitstrings.view(np.int64)).cuda()
        P = int(plan.info["num_paths"])
        pr_end = min(P, args.paths) if args.paths else 0     # profiling aid: a leading path range
        for _ in range(args.warmup):
            plan.run(bits, path_range=(0, pr_end))
        hsf.hsf_set_profiling(True)
        l0 = hsf.hsf_launch_count()
        with ClockSampler(0) as clk:
            ms = _timed(torch, stream, lambda: plan.run(bits, path_range=(0, pr_end)), args.steps)
        launches = hsf.hsf_launch_count() - l0
        st = hsf.hsf_profile_collect(plan.handle)
        hsf.hsf_set_profiling(False)
        line.update({
            "metric": f"HSF circuits/s ({pr.name})", "value": args.steps / (ms / 1e3), "unit": "circuits/s",
            "ms_per_step": ms / args.steps, "dtype": "c64" if args.workload == "c5" else "c128",
            "config": {"workload": pr.name, "n": pr.n, "paths": P,
                       "step": "run only (plan reused)"},
            "gpu_launches": int(launches),
            "kernels": {k: {"launches": int(v["launches"]), "ms": v["ms"]} for k, v in st.items() if v["launches"]},
            "clocks": clk.summary()})
        if pr_end:
            line["config"]["paths_simulated"] = pr_end
            line["value"] = None
            line["est_seconds_all_paths"] = ms / args.steps / 1e3 * P / pr_end
        plan.close()
    print(json.dumps(line), flush=True)


def read_segment_fraction(desc, n, nb, bits):
    """Fraction of the 16-amplitude segments of each half state that the bitstrings'
    chunks fall in (the segments the FP16 level before the leaf contraction stores),
    from the storage order the plan description prints ("side a: h=.. store=[..]")."""
    import re
    fr = []
    for side, m in zip(("a", "b"), re.finditer(r"side ([ab]): h=(\d+) store=\[([0-9,]*)\]", desc)):
        h = int(m.group(2))
        store = [int(x) for x in m.group(3).split(",")]
        x = (bits >> np.uint64(nb)) if m.group(1) == "a" else (bits & np.uint64((1 << nb) - 1))
        idx = np.zeros_like(x)
        for q, t in enumerate(store):
            idx |= ((x >> np.uint64(q)) & np.uint64(1)) << np.uint64(t)
        fr.append(len(np.unique(idx >> np.uint64(4))) / float(1 << (h - 4)))
    return fr


def form_leg(hsf, torch, pr, bits, S, stream, steps, flags, gold, budget):
    """Plan + run of the whole circuit `steps` times with the given plan flags: circuits/s,
    run-only circuits/s and the max error of the output against the stored FP64 values."""
    plan = hsf.Plan.from_problem(pr, precision="c64", flags=flags)
    desc = hsf.hsf_plan_describe(plan.handle)
    need = hsf.hsf_workspace_size(plan.handle, S, 0, budget)
    ws = torch.empty(need, dtype=torch.uint8, device=bits.device)
    out = torch.empty(S, dtype=torch.complex128, device=bits.device)

    def step(h):
        hsf.hsf_run(h, bits.data_ptr(), S, 0, 0, 0, out.data_ptr(), ws.data_ptr(), need, stream.cuda_stream)

    marsh = hsf.Marshalled(pr.n, pr.gates, pr.blocks)

    def full():
        h = hsf.hsf_plan_create(pr.n, pr.gates, pr.cut, pr.blocks, precision="c64", flags=flags, marshalled=marsh)
        step(h)
        return h

    for h in [full() for _ in range(2)]:
        torch.cuda.synchronize()
        hsf.hsf_plan_destroy(h)
    handles = []
    ms = _timed(torch, stream, lambda: handles.append(full()), steps)
    for h in handles:
        hsf.hsf_plan_destroy(h)
    ms_run = _timed(torch, stream, lambda: step(plan.handle), steps)
    hsf.hsf_sync(plan.handle, stream.cuda_stream)
    err = float(np.max(np.abs(out.cpu().numpy() - gold["amps"])))
    tc = sorted({int(l.split()[1].rstrip(":")) for l in desc.splitlines()
                 if l.startswith(" level ") and "tensor-core product" in l})
    plan.close()
    return {"value": steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "run_only_ms": ms_run / steps, "err_vs_fp64": err, "tensor_core_levels": tc,
            "flags": int(flags)}


def path_gemm_leg(hsf, torch, g3):
    """The window path GEMM of the largest 64-batch circuit (n = 32, 4096 paths, leading
    2^24 amplitudes), split-BF16 on the tensor cores and FP32 on the CUDA cores, timed with
    per-kernel events; errors at the stored oracle samples of the window."""
    from paper_2502_06959_gb300 import workloads as W
    pr = W.workload_c3_largest()
    window = int(g3["window"])
    idx = torch.from_numpy(np.array(g3["indices"], dtype=np.int64)).cuda()
    hbm_peak, bf16_peak, sm_max, peak_src = peaks()
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
    res = {"kernel": "path_gemm", "circuit": pr.name, "n": pr.n, "window": window}
    for gemm in ("bf16x3", "fp32"):
        plan = hsf.Plan.from_problem(pr, precision="c64", gemm=gemm)
        out = plan.run(window=window, check=True)
        hsf.hsf_set_profiling(True)
        plan.run(window=window, out=out)
        torch.cuda.synchronize()
        st = hsf.hsf_profile_collect(plan.handle)
        hsf.hsf_set_profiling(False)
        w = st["window"]
        pk = st.get("pack", {"ms": 0.0})
        P = int(plan.info["num_paths"])
        M, N = -(-window // (1 << (pr.cut + 1))), min(window, 1 << (pr.cut + 1))
        useful = 8.0 * M * N * P
        err = float(np.max(np.abs(out[idx].cpu().numpy() - g3["amps"])))
        tfl = w["flops"] / (w["ms"] / 1e3) / 1e12 if w["ms"] else 0.0
        r = {"ms": w["ms"], "pack_ms": pk["ms"], "paths": P, "M": M, "N": N,
             "useful_complex_tflops": useful / (w["ms"] / 1e3) / 1e12,
             "err_vs_fp64": err, "err_samples": int(idx.numel())}
        if gemm == "bf16x3":
            r.update({"bound": "tensor", "achieved": tfl, "peak": bf16_peak, "unit": "TFLOP/s",
                      "frac": tfl / bf16_peak, "traffic": None,
                      "peak_source": peak_src + " (bf16 dense; counted flops = 3 bf16 products per MAC term)"})
        else:
            r.update({"bound": "alu", "achieved": tfl, "peak": fp32_peak, "unit": "TFLOP/s", "frac": tfl / fp32_peak,
                      "peak_source": "152 SMs x 128 FP32 lanes x 2 x max SM clock"})
        res[gemm] = r
        plan.close()
    res.update({k: res["bf16x3"][k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")})
    return res


def sbm_leg(hsf, torch, steps):
    """Table I on one GPU for a q30-1-shaped instance (single-layer QAOA on a 15|15
    stochastic-block-model graph, p_intra 0.8, p_inter 0.1; the first 10^6 amplitudes):
    joint cut with the library's own blocks (hsf_find_blocks), the standard per-gate cut
    (a leading path sample, extrapolated) and the full-state Schroedinger plan, each
    plan + run.  The paper's CPU numbers for q30-1 are context only."""
    from paper_2502_06959_gb300 import workloads as W
    pr = W.sbm_qaoa((15, 15), 0.8, 0.1, seed=1)
    q = hsf.problem_with_found_blocks(pr)
    window = 10 ** 6
    out = torch.empty(window, dtype=torch.complex128, device="cuda")

    def timed_plan_run(make, path_end=0, reps=steps):
        plan = make()
        plan.run(window=window, out=out, path_range=(0, path_end), check=True)   # workspace + warm-up
        ws = plan.workspace(0, window)
        plan.close()
        st = torch.cuda.current_stream()
        handles = []

        def one():
            p = make()
            hsf.hsf_run(p.handle, 0, 0, window, 0, path_end, out.data_ptr(), ws.data_ptr(), ws.numel(),
                        st.cuda_stream)
            handles.append(p)
        ms = _timed(torch, st, one, reps)
        info = dict(handles[0].info)
        for p in handles:
            p.close()
        return ms / reps, info

    jms, jinfo = timed_plan_run(lambda: hsf.Plan.from_problem(q, precision="c64"))
    jout = out.clone()
    sms, _ = timed_plan_run(lambda: hsf.Plan.schrodinger(pr.n, pr.gates, precision="c64"))
    err_js = float((jout - out).abs().max())
    plain = W.Problem(n=q.n, gates=q.gates, cut=q.cut, blocks=W.singleton_blocks(q.n, q.gates, q.cut))
    sample = 1 << 16
    pms, pinfo = timed_plan_run(lambda: hsf.Plan.from_problem(plain, precision="c64"), path_end=sample, reps=2)
    plain_paths = int(pinfo["num_paths"])
    plain_est_ms = pms * plain_paths / sample
    return {"workload": "sbm_qaoa_q30_15x15_pintra0.8_pinter0.1_seed1_first1e6", "window": window,
            "two_qubit_gates": pr.meta["two_qubit_gates"], "sep_cuts": pr.meta["crossing"],
            "blocks_found": len(q.blocks), "hubs": q.meta["hubs"],
            "joint": {"paths": int(jinfo["num_paths"]), "ms": jms},
            "plain": {"paths": plain_paths, "sample_paths": sample, "ms_sample": pms, "est_ms": plain_est_ms},
            "schrodinger": {"ms": sms},
            "s_over_j": sms / jms, "t_over_j": plain_est_ms / jms, "max_abs_joint_vs_schrodinger": err_js,
            "paper_q30_1_cpu": {"paths_joint": 2 ** 11, "paths_standard": 2 ** 17, "s_over_j": 69.857,
                                "t_over_j": 190.950, "hardware": "16-core Threadripper PRO 5955WX (Table I)",
                                "note": "context only: the paper's graph instances are not available"}}


GOLDEN_C4 = os.path.join(ROOT, "tests", "golden", "c4_fd_gradient.json")


def c4_leg(hsf, torch, steps):
    """QAOA n=28 gradients (plan + forward + adjoint through every path, autograd
    Function): gradients/s and the error of the complex64 adjoint against the stored FP64
    central differences of all 8 angles."""
    from paper_2502_06959_gb300 import workloads as W
    pr = W.workload_c4()
    bits = torch.from_numpy(pr.bitstrings.view(np.int64)).cuda()
    theta = torch.tensor(pr.params, dtype=torch.float64, requires_grad=True)
    stream = torch.cuda.current_stream()

    def step():
        amps = hsf.HSFAmplitudes.apply(theta, pr, bits, "c64")
        loss = (amps.abs() ** 2).sum()
        theta.grad = None
        loss.backward()
    for _ in range(2):
        step()
    ms = _timed(torch, stream, step, steps)
    g = theta.grad.detach().numpy()
    out = {"workload": "c4_qaoa_n28_p4_1024bitstrings", "value": steps / (ms / 1e3), "unit": "gradients/s",
           "ms_per_step": ms / steps, "params": int(pr.num_params), "precision": "c64"}
    if os.path.exists(GOLDEN_C4):
        ref = np.array(json.load(open(GOLDEN_C4))["grad_richardson"])
        out["max_abs_err"] = float(np.max(np.abs(g - ref)))
        out["max_rel_err"] = float(np.max(np.abs(g - ref)) / np.max(np.abs(ref)))
        out["ref"] = "tests/golden/c4_fd_gradient.json (FP64 central differences, oracle HSF sum)"
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "c2":
        bench_other(args)
        return
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2502_06959_gb300 import hsf
    hsf.load_library()
    pr = workload(rank)
    dev = torch.device("cuda", torch.cuda.current_device())
    bits_np = pr.bitstrings.astype(np.uint64)
    bits = torch.from_numpy(bits_np.view(np.int64)).to(dev)
    S = bits.numel()
    out = torch.empty(S, dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream()

    # workspace sized once for this circuit
    pflags = hsf.FLAG_LEAF_DOTS if args.leaf_dots else 0
    if args.leaf_dots:
        # the ncu traffic ratios were taken on the stored-children path
        for k in ("level_f16", "leaf"):
            PROFILED_TRAFFIC.pop(k, None)
    plan0 = hsf.Plan.from_problem(pr, precision=args.precision, flags=pflags)
    info = dict(plan0.info)
    free, _ = torch.cuda.mem_get_info()
    budget = int(args.budget_gb * 2 ** 30) if args.budget_gb else int(free * 0.7)
    ws_bytes = hsf.hsf_workspace_size(plan0.handle, S, 0, budget)
    p_end = args.paths if args.paths else 0
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)

    # the circuit's C structs are built once; every step still plans it from them
    # (validation, block products, SVD, programs, table upload)
    marsh = hsf.Marshalled(pr.n, pr.gates, pr.blocks)

    def step(plan_each=True):
        if plan_each:
            h = hsf.hsf_plan_create(pr.n, pr.gates, pr.cut, pr.blocks, precision=args.precision, flags=pflags,
                                       marshalled=marsh)
        else:
            h = plan0.handle
        hsf.hsf_run(h, bits.data_ptr(), S, 0, 0, p_end, out.data_ptr(), ws.data_ptr(), ws_bytes,
                    stream.cuda_stream)
        return h

    def sync_all():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    handles = []
    for _ in range(args.warmup):
        handles.append(step())
    torch.cuda.synchronize()
    for h in handles:
        hsf.hsf_plan_destroy(h)
    handles = []

    # ---- timed region: K full steps (plan + run) ----
    sync_all()
    l0 = hsf.hsf_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            handles.append(step())
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = hsf.hsf_launch_count() - l0
    for h in handles:
        hsf.hsf_plan_destroy(h)
    handles = []

    # ---- profiled pass over the same K steps: every launch bracketed by CUDA events on
    # its stream (the library then keeps both halves on one stream, so each pair times
    # one launch alone); gives the per-kernel durations behind the rooflines ----
    hsf.hsf_set_profiling(True)
    sync_all()
    for _ in range(args.steps):
        handles.append(step())
    torch.cuda.synchronize()
    kstats = {}
    for h in handles:
        st = hsf.hsf_profile_collect(h)
        for k, v in st.items():
            acc = kstats.setdefault(k, dict(launches=0, ms=0.0, bytes=0.0, flops=0.0))
            for f in acc:
                acc[f] += v[f]
    hsf.hsf_set_profiling(False)
    for h in handles:
        hsf.hsf_plan_destroy(h)
    handles = []
    ms_t = torch.tensor([ms], device=dev)
    if dist:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms = float(ms_t.item())
    value = args.steps * world / (ms / 1e3)

    # ---- run only (plan reused) ----
    sync_all()
    e0.record(stream)
    for _ in range(args.steps):
        step(plan_each=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_run = e0.elapsed_time(e1)

    # ---- end to end through the C ABI with host buffers ----
    hbits = torch.from_numpy(bits_np.view(np.int64)).pin_memory()
    hout = torch.empty(S, dtype=torch.complex128).pin_memory()
    dbits = torch.empty_like(bits)
    sync_all()
    e0.record(stream)
    for _ in range(args.steps):
        dbits.copy_(hbits, non_blocking=True)
        h = hsf.hsf_plan_create(pr.n, pr.gates, pr.cut, pr.blocks, precision=args.precision, flags=pflags,
                                       marshalled=marsh)
        hsf.hsf_run(h, dbits.data_ptr(), S, 0, 0, p_end, out.data_ptr(), ws.data_ptr(), ws_bytes,
                    stream.cuda_stream)
        hout.copy_(out, non_blocking=True)
        handles.append(h)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1)
    for h in handles:
        hsf.hsf_plan_destroy(h)
    handles = []
    e2e_t = torch.tensor([ms_e2e], device=dev)
    if dist:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_value = args.steps * world / (float(e2e_t.item()) / 1e3)

    hbm_peak, bf16_peak, sm_max, peak_src = peaks()
    fp32_peak_tflops = 152 * 128 * 2 * sm_max * 1e6 / 1e12
    tf32_peak_tflops = bf16_peak * 1.1 / 2.25          # nominal dense TF32 / BF16 ratio
    total_kernel_ms = sum(v["ms"] for v in kstats.values())

    def roofline_of(kind):
        """The kernel against the roof that binds its algorithmic work: the HBM roof when
        its bytes take longer at the measured bandwidth than its FLOP at the compute
        peak of its unit (FP32 ALU; TF32 or FP16 tensor pipe), else that compute roof.
        The other roof's fraction is reported beside it."""
        st = kstats.get(kind, {})
        k_ms, nlk = st.get("ms", 0.0), max(1, st.get("launches", 1))
        gbs = st.get("bytes", 0.0) / (k_ms / 1e3) / 1e9 if k_ms else 0.0
        tfl = st.get("flops", 0.0) / (k_ms / 1e3) / 1e12 if k_ms else 0.0
        tr = traffic_per_launch(kind, st.get("bytes", 0.0) / nlk)
        r = {"kernel": kind, "launches": int(st.get("launches", 0)), "avg_launch_ms": k_ms / nlk,
             "share": k_ms / total_kernel_ms if total_kernel_ms else 0.0}
        if kind == "level_mma":
            # three TF32 products per level: counted flops are the products issued
            cpeak, cunit, csrc = tf32_peak_tflops, "tensor", peak_src + " (bf16 x 1.1/2.25 nominal TF32 ratio)"
        elif kind == "level_f16":
            cpeak, cunit, csrc = bf16_peak, "tensor", peak_src + " (cuBLAS bf16; fp16 has the same nominal dense rate)"
        else:
            cpeak, cunit, csrc = fp32_peak_tflops, "alu", "152 SMs x 128 FP32 lanes x 2 x max SM clock"
        intensity = st.get("flops", 0.0) / st.get("bytes", 1.0) if st.get("bytes") else 0.0
        balance = cpeak * 1e12 / (hbm_peak * 1e9) if hbm_peak else 0.0
        hbm = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak if hbm_peak else None,
               "peak_source": peak_src}
        comp = {"achieved": tfl, "peak": cpeak, "unit": "TFLOP/s", "frac": tfl / cpeak if cpeak else None,
                "peak_source": csrc}
        if intensity < balance:
            r.update({"bound": "hbm", **hbm, "traffic": tr, "flop_per_byte": intensity, "balance": balance,
                      cunit: comp})
        else:
            r.update({"bound": cunit, **comp, "traffic": tr, "flop_per_byte": intensity, "balance": balance,
                      "hbm": hbm})
        return r

    dominant = max(kstats, key=lambda k: kstats[k]["ms"]) if kstats else "sweep"

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {**C2_CONFIG, "n": pr.n, "cut": pr.cut,
                   "paths": int(info["num_paths"]), "tree_nodes_per_side": int(info["tree_nodes"]),
                   "bitstrings": S, "blocks": len(pr.blocks),
                   "l2": "working set (half-state buffers) >> L2, no flush needed",
                   "step": "plan (host + FP64 SVD kernel) + run (all paths)"},
        "gpu_launches": int(launches),
        "run_only": {"value": args.steps / (ms_run / 1e3), "unit": UNIT, "ms_per_step": ms_run / args.steps},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(S * 8),
                "d2h_bytes_per_step": int(S * 16)},
        "roofline": dict(roofline_of(dominant),
                         measured="profiled pass of the same steps, halves on one stream"),
        "rooflines": {k: roofline_of(k) for k in ("sweep", "level_mma", "level_f16", "leaf") if k in kstats},
        "leaf_level_segments_read": read_segment_fraction(hsf.hsf_plan_describe(plan0.handle), pr.n, pr.cut + 1,
                                                          bits_np.astype(np.uint64)),
        "kernels": {k: {"launches": int(v["launches"]), "ms": v["ms"],
                        "share": v["ms"] / total_kernel_ms if total_kernel_ms else 0.0}
                    for k, v in kstats.items() if v["launches"]},
        "clocks": clk.summary(),
    }

    if args.paths:
        line["config"]["paths_simulated"] = args.paths
        line["value"] = None       # a partial path sum is not a circuit
    if rank == 0 and not args.no_extras:
        # joint vs plain cut: the same circuit with one block per crossing gate (2^32
        # paths) timed on a fixed path budget and extrapolated
        from paper_2502_06959_gb300 import workloads as W
        plain_blocks = W.singleton_blocks(pr.n, pr.gates, pr.cut)
        pp = hsf.Plan(pr.n, pr.gates, pr.cut, plain_blocks, precision=args.precision)
        budget_paths = 1 << 16
        pp.run(bits, path_range=(0, budget_paths))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pp.run(bits, path_range=(0, budget_paths))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        plain_paths = int(pp.info["num_paths"])
        est = plain_paths * dt / budget_paths
        line["plain_cut"] = {"paths": plain_paths, "sample_paths": budget_paths,
                             "paths_per_s": budget_paths / dt, "est_seconds": est,
                             "joint_speedup_vs_plain": est / (ms / 1e3 / args.steps)}
        pp.close()
        # CPU oracle baseline on a bounded sample of the same circuit's paths
        cores = cpu_cores()
        ppc = calibrate_paths_per_core(pr, args.cpu_seconds, cores)
        ref, dt, tot = oracle_sample(pr, ppc, cores, start=0)
        P = int(info["num_paths"])
        cpu_value = tot / dt / P
        line["cpu_baseline"] = {"value": cpu_value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"paths [0, {tot}) of {P} on {cores} spawned processes, "
                                          f"{dt:.1f} s, extrapolated to the full path count"}
        # error of the timed steps' output (all 65536 paths) against the stored FP64
        # Schroedinger amplitudes of the same circuit
        gold = load_golden(GOLDEN_C2) if not args.paths else None
        if gold is not None and gold["seed"] == 2 and args.precision == "c64":
            got = out.cpu().numpy()
            line["err_vs_fp64"] = {"max_abs": float(np.max(np.abs(got - gold["amps"]))),
                                   "max_ref": float(np.max(np.abs(gold["amps"]))), "paths": P,
                                   "precision": args.precision,
                                   "ref": "tests/golden/c2_n30_amplitudes.json (FP64 Schroedinger oracle)"}
            # the precision forms on the same circuit: the default (tensor-core levels with
            # FP16 / TF32 split operands) against the plain FP32 path (every level swept on
            # the CUDA cores), each timed over the same steps and checked against FP64; and
            # the opt-in dot form of the leaf (level 7 writes the leaf's chunk dots instead
            # of its children: fewer bytes, a slower epilogue)
            line["forms"] = {
                "default_tc_levels": form_leg(hsf, torch, pr, bits, S, stream, args.steps, 0, gold, budget),
                "plain_fp32": form_leg(hsf, torch, pr, bits, S, stream, args.steps, hsf.FLAG_NO_TC_LEVEL, gold,
                                       budget),
                "leaf_dots": form_leg(hsf, torch, pr, bits, S, stream, args.steps, hsf.FLAG_LEAF_DOTS, gold,
                                      budget),
            }
        else:
            got = plan0.run(bits, path_range=(0, tot)).cpu().numpy()
            line["err_vs_fp64"] = {"max_abs": float(np.max(np.abs(got - ref))), "max_ref": float(np.max(np.abs(ref))),
                                   "paths": tot, "precision": args.precision, "ref": "oracle path sample"}
        g3 = load_golden(GOLDEN_C3)
        if g3 is not None:
            line["rooflines"]["path_gemm"] = path_gemm_leg(hsf, torch, g3)
        # Schroedinger on the same GPU for the benchmark circuit itself (Table I's S/J)
        sch = hsf.Plan.schrodinger(pr.n, pr.gates, precision="c64")
        sch.run(bits, out=out, check=True)
        ws_s = sch.workspace(S, 0)
        hsf.hsf_set_profiling(True)
        sch.run(bits, out=out)
        torch.cuda.synchronize()
        sst = hsf.hsf_profile_collect(sch.handle)["sweep"]
        hsf.hsf_set_profiling(False)
        s_passes = int(sch.info["num_launches"])
        sch.close()
        hs = []

        def sch_step():
            h = hsf.hsf_plan_create_schrodinger(pr.n, pr.gates, precision="c64")
            hsf.hsf_run(h, bits.data_ptr(), S, 0, 0, 0, out.data_ptr(), ws_s.data_ptr(), ws_s.numel(),
                        stream.cuda_stream)
            hs.append(h)
        ms_s = _timed(torch, stream, sch_step, 2)
        for h in hs:
            hsf.hsf_plan_destroy(h)
        del ws_s
        serr = float(np.max(np.abs(out.cpu().numpy() - gold["amps"]))) if gold is not None else None
        fp32_peak = 152 * 128 * 2 * peaks()[2] * 1e6 / 1e12
        line["schrodinger"] = {"ms_per_step": ms_s / 2, "s_over_j": (ms_s / 2) / (ms / args.steps),
                               "err_vs_fp64": serr, "state": "2^30 complex64 (8 GB)", "passes": s_passes,
                               "sweep_ms": sst["ms"], "sweep_gbs": sst["bytes"] / (sst["ms"] / 1e3) / 1e9,
                               "sweep_tflops": sst["flops"] / (sst["ms"] / 1e3) / 1e12,
                               "sweep_alu_frac": sst["flops"] / (sst["ms"] / 1e3) / 1e12 / fp32_peak,
                               "step": "plan + full-state sweep + read-out"}
        line["sbm_table1"] = sbm_leg(hsf, torch, args.steps)
        line["c4"] = c4_leg(hsf, torch, args.steps)
    plan0.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
