"""Path sharding through the library: two ranks (gloo, both on cuda:0) each run hsf_run
over their subtree range of the paths (Sec. II-B: the paths are independent), and the
all-reduced partial sums equal the single-rank run and the FP64 oracle.

The ranks share one GPU but nothing on it waits for the other rank: each runs its own
kernels to completion, and the sum-reduce goes through host memory with gloo."""
import os

import numpy as np
import pytest

from paper_2502_06959_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _problem():
    pr = W.random_brickwork(20, 9, 6, block_after=(1, 3, 5), block_kind="mixed", block_len=3, seed=17)
    bits = W.random_bitstrings(np.random.default_rng(17), pr.n, 512)
    return pr, bits


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_2502_06959_gb300 import hsf, sharding
    hsf.load_library()
    pr, bits = _problem()
    b = torch.from_numpy(bits.view(np.int64)).cuda()
    plan = hsf.Plan.from_problem(pr, precision="c128")
    out = sharding.run_sharded(plan, b, rank, world).cpu().numpy()
    if rank == 0:
        full = plan.run(b).cpu().numpy()
        q.put((out, full, int(plan.info["num_paths"])))
    plan.close()
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_sharded_hsf_run_equals_single_run_and_oracle():
    import torch.multiprocessing as mp
    import oracle.hsf_oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 31500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=300)
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out, full, P = res
    assert P > 2
    assert np.max(np.abs(out - full)) <= 1e-13
    pr, bits = _problem()
    ref = O.schrodinger(pr.n, pr.gates)[bits.astype(np.int64)]
    assert np.max(np.abs(out - ref)) <= 1e-12
