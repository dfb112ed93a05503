"""Write tests/golden/c3_largest_window.json: FP64 amplitudes of the largest circuit of the
64-circuit batch (n = 32, 6 blocks, 4^6 = 4096 joint paths) at 4096 seeded indices of its
leading window of 2^24 amplitudes.

The values come from the oracle's HSF path sum over all paths (oracle.hsf_amplitudes,
Sec. II-B), which the CPU tests pin to the plain Schroedinger oracle; the full n = 32
statevector (64 GB) does not fit this host.  Inputs come from the seeded generator
(paper_2502_06959_gb300.workloads), which holds none of the method's arithmetic.

    python tests/golden/make_c3_golden.py      # about ten minutes on 8 cores
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

OUT = os.path.join(HERE, "c3_largest_window.json")
WINDOW = 1 << 24
SAMPLES = 4096
SAMPLE_SEED = 33


def _part(args):
    sys.path.insert(0, ROOT)
    import oracle.hsf_oracle as O
    from paper_2502_06959_gb300 import workloads as W
    a, b, idx = args
    pr = W.workload_c3_largest()
    out, info = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=idx, path_range=(a, b))
    return out, info["num_paths"]


def main():
    from paper_2502_06959_gb300 import workloads as W
    pr = W.workload_c3_largest()
    idx = W.window_samples(pr.n, WINDOW, SAMPLES, SAMPLE_SEED)
    import oracle.hsf_oracle as O
    dec = O.decompose_blocks(pr.n, pr.gates, pr.cut, pr.blocks)
    P = int(np.prod([len(d["sigma"]) for d in dec]))
    cores = os.cpu_count() or 1
    edges = np.linspace(0, P, cores + 1).astype(int)
    # one BLAS thread per worker process: the pool already uses every core
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    t0 = time.time()
    with mp.get_context("spawn").Pool(cores) as pool:
        parts = pool.map(_part, [(int(edges[i]), int(edges[i + 1]), idx) for i in range(cores)])
    amps = np.sum([p[0] for p in parts], axis=0)
    dt = time.time() - t0
    rec = {
        "what": "amplitudes of the largest 64-batch circuit at seeded indices of its leading 2^24 window",
        "cite": "Sec. II-B (sum over all paths of the two halves' Kronecker products); Sec. V (leading window)",
        "generator": "paper_2502_06959_gb300.workloads.workload_c3_largest + window_samples",
        "name": pr.name, "n": pr.n, "cut": pr.cut, "num_gates": len(pr.gates), "num_blocks": len(pr.blocks),
        "paths": P, "window": WINDOW, "sample_seed": SAMPLE_SEED,
        "script": "tests/golden/make_c3_golden.py (oracle.hsf_amplitudes, FP64, all paths)",
        "seconds": round(dt, 1), "max_abs": float(np.max(np.abs(amps))),
        "indices": [int(i) for i in idx],
        "re": [float(a.real) for a in amps],
        "im": [float(a.imag) for a in amps],
    }
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=0)
    print(f"wrote {OUT}: {len(idx)} amplitudes over {P} paths, {dt:.0f} s")


if __name__ == "__main__":
    main()
