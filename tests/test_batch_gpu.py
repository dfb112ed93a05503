"""Batches in one CUDA graph and the autotuner (GPU)."""
import os
import tempfile

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


def test_graph_batch_of_uneven_circuits_matches_single_runs_and_oracle():
    import torch
    from paper_2502_06959_gb300 import hsf
    rng = np.random.default_rng(5)
    items, refs = [], []
    for i, n in enumerate((8, 12, 10, 14, 9, 12)):
        pr = W.random_brickwork(n, n // 2 - 1, 5, block_after=tuple(sorted(rng.choice(5, 2, replace=False) + 1)),
                                block_kind="mixed", block_len=3, seed=50 + i)
        ref = O.schrodinger(pr.n, pr.gates)
        gemm = ("fp32", "bf16x3", "tf32x3")[i % 3]
        plan = hsf.Plan.from_problem(pr, precision="c64", gemm=gemm)
        if i % 2 == 0:
            window = min(1 << n, 700)
            out = torch.zeros(window, dtype=torch.complex128, device="cuda")
            items.append(dict(plan=plan, window=window, out=out))
            refs.append(ref[:window])
        else:
            bits = W.random_bitstrings(rng, n, 100)
            b = torch.from_numpy(bits.view(np.int64)).cuda()
            out = torch.zeros(100, dtype=torch.complex128, device="cuda")
            items.append(dict(plan=plan, bitstrings=b, out=out))
            refs.append(ref[bits.astype(np.int64)])
    batch = hsf.Batch(items)
    assert batch.nodes > len(items)
    for rep in range(2):
        for it in items:
            it["out"].fill_(complex(3.0, 3.0))
        batch.launch()
        torch.cuda.synchronize()
        for it, ref in zip(items, refs):
            got = it["out"].cpu().numpy()
            assert np.max(np.abs(got - ref)) <= 1e-5
            assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))
    batch.close()
    for it in items:
        it["plan"].close()


def test_autotuner_picks_a_valid_configuration_and_caches_it():
    import torch
    from paper_2502_06959_gb300 import hsf
    pr = W.random_brickwork(16, 7, 6, block_after=(2, 4), block_kind="mixed", block_len=3, seed=9)
    bits = W.random_bitstrings(np.random.default_rng(0), pr.n, 64)
    b = torch.from_numpy(bits.view(np.int64)).cuda()
    with tempfile.TemporaryDirectory() as d:
        cache = os.path.join(d, "tune.txt")
        opts = hsf.hsf_tune(pr.n, pr.gates, pr.cut, pr.blocks, num=64, bitstrings_ptr=b.data_ptr(),
                            cache_path=cache)
        assert 3 <= opts["tile_bits"] <= 13
        assert os.path.getsize(cache) > 0
        again = hsf.hsf_tune(pr.n, pr.gates, pr.cut, pr.blocks, num=64, bitstrings_ptr=b.data_ptr(),
                             cache_path=cache)
        assert again == opts
        assert len(open(cache).read().splitlines()) == 1
    plan = hsf.Plan.from_problem(pr, tile_bits=opts["tile_bits"], flags=opts["flags"])
    got = plan.run(b).cpu().numpy()
    plan.close()
    ref = O.schrodinger(pr.n, pr.gates)[bits.astype(np.int64)]
    assert np.max(np.abs(got - ref)) <= 1e-5
