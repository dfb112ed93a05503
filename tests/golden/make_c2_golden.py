"""Write tests/golden/c2_n30_amplitudes.json: FP64 amplitudes of the n=30 joint-cut
benchmark circuit at its 4096 seeded bitstrings.

The values come from the plain Schroedinger oracle alone (oracle/schrodinger.c: one
gate at a time on the full 2^30 statevector, Sec. II-A), never from the CUDA path; the
circuit and bitstrings come from the seeded input generator
(paper_2502_06959_gb300.workloads.workload_c2, seed 2), which draws inputs only.

Needs 16 GB of host memory and about half an hour on 8 cores:
    python tests/golden/make_c2_golden.py
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle.schrodinger_c import schrodinger_c          # noqa: E402
from paper_2502_06959_gb300 import workloads as W       # noqa: E402

OUT = os.path.join(HERE, "c2_n30_amplitudes.json")


def main():
    seed = 2
    pr = W.workload_c2(seed=seed)
    t0 = time.time()
    psi = schrodinger_c(pr.n, pr.gates)
    dt = time.time() - t0
    norm = float(np.sqrt(np.vdot(psi, psi).real))
    bits = pr.bitstrings.astype(np.uint64)
    amps = psi[bits.astype(np.int64)]
    rec = {
        "what": "amplitudes <x|U|0...0> of the n=30 joint-cut benchmark circuit at its seeded bitstrings",
        "cite": "Sec. II-A (Schroedinger simulation: consecutive gate applications on the full statevector)",
        "generator": "paper_2502_06959_gb300.workloads.workload_c2",
        "seed": seed, "n": pr.n, "cut": pr.cut, "num_gates": len(pr.gates), "num_blocks": len(pr.blocks),
        "script": "tests/golden/make_c2_golden.py (oracle/schrodinger.c, FP64)",
        "seconds": round(dt, 1), "norm": norm,
        "max_abs": float(np.max(np.abs(amps))),
        "bitstrings": [int(b) for b in bits],
        "re": [float(a.real) for a in amps],
        "im": [float(a.imag) for a in amps],
    }
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=0)
    print(f"wrote {OUT}: {len(bits)} amplitudes, norm {norm:.15f}, {dt:.0f} s")


if __name__ == "__main__":
    main()
