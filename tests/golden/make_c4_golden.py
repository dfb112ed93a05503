"""Write tests/golden/c4_fd_gradient.json: the FP64 central-difference gradient of the
QAOA loss L = sum_s |amp(s)|^2 (n = 28, p = 4, 1024 seeded bitstrings, both ring edges
crossing the cut jointly cut per layer) with respect to all 8 angles.

Every loss value comes from the oracle's HSF path sum (oracle.hsf_amplitudes, Sec. II-B),
which the CPU tests pin to the Schroedinger oracle; the differences use steps h and h/2
so that the stored Richardson gap bounds the O(h^2) error.  Inputs come from the seeded
generator (paper_2502_06959_gb300.workloads.workload_c4).

    python tests/golden/make_c4_golden.py
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "c4_fd_gradient.json")
H = 1e-4


def _loss(theta):
    sys.path.insert(0, ROOT)
    import oracle.hsf_oracle as O
    from paper_2502_06959_gb300 import workloads as W
    pr = W.workload_c4()
    amps, _ = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=pr.bitstrings, theta=theta)
    return O.loss_from_amplitudes(amps)


def main():
    from paper_2502_06959_gb300 import workloads as W
    pr = W.workload_c4()
    th = np.asarray(pr.params, dtype=np.float64)
    jobs = [th.copy()]
    for h in (H, H / 2):
        for j in range(th.size):
            for sgn in (1, -1):
                t = th.copy()
                t[j] += sgn * h
                jobs.append(t)
    # one BLAS thread per worker process: the pool already uses every core
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    t0 = time.time()
    with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        vals = pool.map(_loss, jobs)
    dt = time.time() - t0
    loss0 = vals[0]
    v = np.array(vals[1:]).reshape(2, th.size, 2)
    g_h = (v[0, :, 0] - v[0, :, 1]) / (2 * H)
    g_h2 = (v[1, :, 0] - v[1, :, 1]) / H
    rich = (4 * g_h2 - g_h) / 3
    rec = {
        "what": "FP64 central-difference gradient of sum_s |amp(s)|^2 for the n=28 QAOA workload",
        "cite": "Sec. II-B (HSF path sum for every loss value); central differences, Richardson check",
        "generator": "paper_2502_06959_gb300.workloads.workload_c4",
        "script": "tests/golden/make_c4_golden.py (oracle.hsf_amplitudes, FP64)",
        "h": H, "seconds": round(dt, 1), "loss": loss0, "theta": th.tolist(),
        "grad_h": g_h.tolist(), "grad_h2": g_h2.tolist(), "grad_richardson": rich.tolist(),
        "fd_error_bound": float(np.max(np.abs(g_h2 - rich))),
    }
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
    print(f"wrote {OUT}: loss {loss0:.6e}, max |g| {np.max(np.abs(rich)):.3e}, "
          f"h/2 vs Richardson {rec['fd_error_bound']:.2e}, {dt:.0f} s")


if __name__ == "__main__":
    main()
