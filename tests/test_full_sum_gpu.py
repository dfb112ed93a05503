"""The whole path sum of the n = 30 benchmark circuit against stored FP64 amplitudes.

tests/golden/c2_n30_amplitudes.json holds <x|U|0...0> at the circuit's 4096 seeded
bitstrings, written by tests/golden/make_c2_golden.py from the plain Schroedinger
oracle (one gate at a time on the full 2^30 statevector, Sec. II-A).  Here the CUDA path
sums all 4^8 = 65536 joint paths (Sec. II-B) in the benchmark's launch configuration:
FP16-split tensor-core product at tree level 7, TF32-split products with epilogue ops at
levels 5 and 6, CUDA-core sweeps above, the grouped leaf contraction at the bitstrings
and the FP64 Neumaier reduction over parent groups and path chunks.  The bound is the
complex64 one: 1e-5 absolute and 1e-4 of the largest reference amplitude.  complex128
half states (no tensor-core levels) are held to 1e-12, where FP64 is kept end to end.
"""
import json
import os

import numpy as np
import pytest

from paper_2502_06959_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c2_n30_amplitudes.json")


@pytest.fixture(scope="module")
def golden():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2502_06959_gb300 import build
    build.build()
    from paper_2502_06959_gb300 import hsf
    hsf.load_library()
    with open(GOLDEN) as f:
        rec = json.load(f)
    pr = W.workload_c2(seed=rec["seed"])
    bits = np.array(rec["bitstrings"], dtype=np.uint64)
    assert np.array_equal(bits, pr.bitstrings.astype(np.uint64)), "generator drifted from the stored bitstrings"
    assert len(pr.gates) == rec["num_gates"]
    ref = np.array(rec["re"]) + 1j * np.array(rec["im"])
    assert abs(rec["norm"] - 1.0) < 1e-12
    return pr, bits, ref


def _run(pr, bits, precision="c64", budget=0, **opts):
    import torch
    from paper_2502_06959_gb300 import hsf
    plan = hsf.Plan.from_problem(pr, precision=precision, **opts)
    desc = hsf.hsf_plan_describe(plan.handle)
    dbits = torch.from_numpy(bits.view(np.int64)).cuda()
    S = bits.size
    free, _ = torch.cuda.mem_get_info()
    full = hsf.hsf_workspace_size(plan.handle, S, 0, int(free * 0.7))
    need = hsf.hsf_workspace_size(plan.handle, S, 0, budget) if budget else full
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    out = torch.empty(S, dtype=torch.complex128, device="cuda")
    st = torch.cuda.current_stream()
    hsf.hsf_run(plan.handle, dbits.data_ptr(), S, 0, 0, 0, out.data_ptr(), ws.data_ptr(), need, st.cuda_stream)
    hsf.hsf_sync(plan.handle, st.cuda_stream)
    got = out.cpu().numpy()
    info = dict(plan.info)
    plan.close()
    return got, desc, info, need, full


def _check_c64(got, ref):
    err = float(np.max(np.abs(got - ref)))
    scale = float(np.max(np.abs(ref)))
    assert err <= 1e-5, err
    assert err <= 1e-4 * scale, (err, scale)
    return err


def test_all_paths_benchmark_kernels(golden):
    pr, bits, ref = golden
    got, desc, info, _, _ = _run(pr, bits)
    assert info["num_paths"] == 4 ** 8
    assert info["leaf_bits"] > 0, "the leaf level is contracted at the bitstrings"
    for lvl, kind in ((7, "product (FP16x3)"), (6, "product (TF32x3)"), (5, "product (TF32x3)")):
        lines = [l for l in desc.splitlines() if l.startswith(f" level {lvl}:")]
        assert len(lines) == 2 and all(kind in l for l in lines), (lvl, desc)
    for lvl in (5, 6):
        lines = [l for l in desc.splitlines() if l.startswith(f" level {lvl}:")]
        assert all("ops in its epilogue" in l for l in lines), (lvl, desc)
    _check_c64(got, ref)


def test_all_paths_several_chunks(golden):
    """A workspace budget that holds an eighth of the full layout: the path tree is
    walked in several subtree chunks, each refolded into the FP64 output."""
    pr, bits, ref = golden
    import torch
    from paper_2502_06959_gb300 import hsf
    plan = hsf.Plan.from_problem(pr)
    free, _ = torch.cuda.mem_get_info()
    full = hsf.hsf_workspace_size(plan.handle, bits.size, 0, int(free * 0.7))
    plan.close()
    got, _, _, need, _ = _run(pr, bits, budget=full // 8)
    assert need < full
    _check_c64(got, ref)


def test_all_paths_cuda_cores(golden):
    """The plain FP32 path (every tree level swept on the CUDA cores) at the same bound."""
    from paper_2502_06959_gb300 import hsf
    pr, bits, ref = golden
    got, desc, _, _, _ = _run(pr, bits, flags=hsf.FLAG_NO_TC_LEVEL)
    assert "tensor-core product" not in desc
    _check_c64(got, ref)


def test_all_paths_complex128(golden):
    """FP64 half states and FP64 sums: the whole 65536-path sum within 1e-12."""
    pr, bits, ref = golden
    got, desc, _, _, _ = _run(pr, bits, precision="c128")
    err = float(np.max(np.abs(got - ref)))
    assert err <= 1e-12, err


@pytest.mark.parametrize("count", [1, 37, 512])
def test_all_paths_few_bitstrings(golden, count):
    """Few bitstrings: level 7 then stores only the 16-amplitude segments that those
    bitstrings' chunks cover (almost none of the state at one bitstring), and the leaf
    must still see exactly the values it reads.  The first `count` stored bitstrings,
    all 65536 paths, against the same FP64 amplitudes; the plan is the benchmark's
    (FP16 level 7 before the factored leaf)."""
    pr, bits, ref = golden
    got, desc, _, _, _ = _run(pr, bits[:count].copy())
    assert "leaf=factored" in desc
    assert any(l.startswith(" level 7:") and "FP16x3" in l for l in desc.splitlines())
    # the same bound as the full set (1e-5 absolute, 1e-4 of the largest of the 4096
    # reference amplitudes): the error does not depend on which bitstrings are asked
    err = float(np.max(np.abs(got - ref[:count])))
    assert err <= 1e-5 and err <= 1e-4 * float(np.max(np.abs(ref))), err
