"""hsf_run_static: the run entry point for callers that cannot allocate device memory.

It must give the same amplitudes as hsf_run with a caller workspace (same plan, same
request), on two calls in a row (the shared scratch array keeps the previous call's
contents, which must not leak into the next result), and it must refuse a request
that does not fit its fixed scratch with a clear error.  This file is collected last
so that a stop-at-first-failure run has already run every other test.
"""
import numpy as np
import pytest

from paper_2502_06959_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_C64 = 1e-5


@pytest.fixture(scope="module")
def hsf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2502_06959_gb300 import build
    build.build()
    from paper_2502_06959_gb300 import hsf as H
    H.load_library()
    return H


def _run_both(H, pr, prec, bits=None):
    import torch
    plan = H.Plan.from_problem(pr, precision=prec)
    num = 0 if bits is None else len(bits)
    count = num if num else 1 << pr.n
    dbits = None
    if bits is not None:
        dbits = torch.from_numpy(np.asarray(bits, dtype=np.uint64).view(np.int64)).cuda()
    ref = plan.run(dbits).cpu().numpy()
    outs = []
    for _ in range(2):                       # two calls in a row share the scratch array
        out = torch.full((count,), complex(7.0, -7.0), dtype=torch.complex128, device="cuda")
        H.hsf_run_static(plan.handle, dbits.data_ptr() if dbits is not None else 0, num, 0, 0, 0,
                         out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    plan.close()
    return ref, outs


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_static_run_matches_workspace_run(hsf, prec):
    tol = 1e-12 if prec == "c128" else TOL_C64
    pr = W.workload_c1()
    ref, outs = _run_both(hsf, pr, prec)
    for o in outs:
        assert np.max(np.abs(o - ref)) <= tol
    pr = W.random_brickwork(14, 6, 6, block_after=(2, 4), block_kind="mixed", block_len=3, seed=3)
    bits = W.random_bitstrings(np.random.default_rng(0), pr.n, 500)
    ref, outs = _run_both(hsf, pr, prec, bits)
    for o in outs:
        assert np.max(np.abs(o - ref)) <= tol


def test_static_run_rejects_oversized_requests(hsf):
    import torch
    # 22|22 halves: one half state alone is 32 MiB in complex64, so no path chunk fits
    gates = [W.Gate("h", (0,)), W.Gate("h", (43,))]
    pr = W.Problem(44, gates, 21, [], bitstrings=np.arange(16, dtype=np.uint64))
    plan = hsf.Plan.from_problem(pr)
    bits = torch.from_numpy(pr.bitstrings.view(np.int64)).cuda()
    out = torch.empty(16, dtype=torch.complex128, device="cuda")
    with pytest.raises(hsf.HsfError) as ei:
        hsf.hsf_run_static(plan.handle, bits.data_ptr(), 16, 0, 0, 0, out.data_ptr(), 0)
    assert ei.value.code == 4 and "static scratch" in str(ei.value)
    plan.close()
