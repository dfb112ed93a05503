"""GPU Schroedinger simulation (hsf_plan_create_schrodinger + hsf_run) against the oracle.

The plan sweeps the full 2^n statevector with the same kernels as the half states
(Sec. II-A; the method Table I's column S times).  Checked against the numpy oracle
(n <= 20), the C oracle (n = 24) and the stored n = 30 benchmark amplitudes; complex128
within 1e-12, complex64 within 1e-5 absolute and 1e-4 of the largest amplitude.
"""
import json
import os

import numpy as np
import pytest

import oracle.hsf_oracle as O
from paper_2502_06959_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2502_06959_gb300 import build
    build.build()
    from paper_2502_06959_gb300 import hsf
    hsf.load_library()


TOL = {"c128": 1e-12, "c64": 1e-5}


def _run(n, gates, precision, bits=None, window=0, **opts):
    import torch
    from paper_2502_06959_gb300 import hsf
    plan = hsf.Plan.schrodinger(n, gates, precision=precision, **opts)
    info = dict(plan.info)
    b = None if bits is None else torch.from_numpy(np.asarray(bits, dtype=np.uint64).view(np.int64)).cuda()
    out = plan.run(b, window=window, check=True).cpu().numpy()
    plan.close()
    return out, info


def _check(got, want, precision):
    err = float(np.max(np.abs(got - want)))
    assert err <= TOL[precision], (precision, err)
    if precision == "c64":
        assert err <= 1e-4 * float(np.max(np.abs(want))), err


@pytest.mark.parametrize("precision", ["c128", "c64"])
@pytest.mark.parametrize("n,seed", [(2, 1), (5, 2), (11, 3), (13, 4), (17, 5)])
def test_random_circuits_full_state(n, seed, precision):
    gates = W.random_circuit(n, 12 * n, seed=seed)
    want = O.schrodinger(n, gates)
    got, info = _run(n, gates, precision)
    assert info["num_paths"] == 1
    _check(got, want, precision)


@pytest.mark.parametrize("precision", ["c128", "c64"])
def test_brickwork_bitstrings_and_window(precision):
    pr = W.random_brickwork(20, 9, 6, block_after=(2, 4), block_kind="mixed", block_len=3, seed=12)
    want = O.schrodinger(pr.n, pr.gates)
    rng = np.random.default_rng(3)
    bits = W.random_bitstrings(rng, pr.n, 777)
    got, _ = _run(pr.n, pr.gates, precision, bits=bits)
    _check(got, want[bits.astype(np.int64)], precision)
    got, _ = _run(pr.n, pr.gates, precision, window=300001)
    _check(got, want[:300001], precision)


def test_three_qubit_gates_and_unfused_sweep():
    from paper_2502_06959_gb300 import hsf
    rng = np.random.default_rng(8)
    z = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
    q, r = np.linalg.qr(z)
    m3 = q * (np.diag(r) / np.abs(np.diag(r)))
    gates = W.random_circuit(16, 100, seed=9)
    gates.insert(40, W.Gate("matrix", (15, 3, 9), matrix=m3))
    want = O.schrodinger(16, gates)
    for flags in (0, hsf.FLAG_NO_REGISTER_SWEEP):
        got, _ = _run(16, gates, "c128", flags=flags)
        _check(got, want, "c128")


def test_n24_against_c_oracle():
    from oracle.schrodinger_c import schrodinger_c
    pr = W.random_brickwork(24, 11, 8, block_after=(2, 5), block_kind="rzz", block_len=3, seed=4)
    want = schrodinger_c(pr.n, pr.gates)
    got, _ = _run(pr.n, pr.gates, "c64")
    _check(got, want, "c64")


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_n30_benchmark_circuit_against_golden(precision):
    path = os.path.join(os.path.dirname(__file__), "golden", "c2_n30_amplitudes.json")
    rec = json.load(open(path))
    pr = W.workload_c2(seed=rec["seed"])
    bits = np.array(rec["bitstrings"], dtype=np.uint64)
    ref = np.array(rec["re"]) + 1j * np.array(rec["im"])
    got, _ = _run(pr.n, pr.gates, precision, bits=bits)
    _check(got, ref, precision)


def test_rejects_too_large_and_bad_input():
    from paper_2502_06959_gb300 import hsf
    with pytest.raises(hsf.HsfError):
        hsf.hsf_plan_create_schrodinger(35, [], precision="c64")
    with pytest.raises(hsf.HsfError):
        hsf.hsf_plan_create_schrodinger(4, [W.Gate("cx", (1, 4))])
