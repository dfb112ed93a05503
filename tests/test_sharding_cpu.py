"""Path sharding across ranks: ranges partition the paths along subtrees, and the
per-rank partial sums reduced with a gloo all-reduce (world size 2, CPU) equal the
single-process sum.  The partial sums come from the FP64 oracle here; on GPUs each
rank would run hsf_run on its range."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2502_06959_gb300 import sharding as S
from paper_2502_06959_gb300 import workloads as W


def test_path_ranges_partition_on_subtrees():
    for P, world, sub in ((4 ** 8, 2, 4 ** 6), (4 ** 8, 3, 4 ** 6), (100, 4, 1), (16, 8, 4), (7, 3, 1)):
        rs = S.path_ranges(P, world, sub)
        assert rs[0][0] == 0 and rs[-1][1] == P
        for (a, b), (c, d) in zip(rs[:-1], rs[1:]):
            assert b == c and a <= b
        if P % sub == 0:
            assert all(a % sub == 0 for a, _ in rs)
    assert S.subtree_size([4] * 8, 2) == 4 ** 7
    assert S.subtree_size([2, 3, 4], 4) == 4


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import oracle.hsf_oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pr = W.random_brickwork(10, 4, 5, block_after=(1, 3, 5), block_kind="mixed", block_len=3, seed=4)
    bits = W.random_bitstrings(np.random.default_rng(0), pr.n, 64)
    _, info = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=bits, path_range=(0, 0))
    sub = S.subtree_size(info["ranks"], world)
    lo, hi = S.path_ranges(info["num_paths"], world, sub)[rank]
    part, _ = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=bits, path_range=(lo, hi))
    t = torch.from_numpy(part.copy())
    S.allreduce_amplitudes(t)
    if rank == 0:
        full, _ = O.hsf_amplitudes(pr.n, pr.gates, pr.cut, pr.blocks, bitstrings=bits)
        q.put(float(np.max(np.abs(t.numpy() - full))))
    dist.destroy_process_group()


def test_gloo_world2_sharded_sum_equals_full_sum():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert q.get(timeout=10) < 1e-13
