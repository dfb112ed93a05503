"""Path sharding of one circuit across ranks (one process per GPU).

The HSF amplitude is a sum over independent paths (Sec. II-B: the paths can be
simulated in parallel), so a circuit is split across G ranks by path ranges and the
partial sums are added with one sum-reduce of the FP64 output.  Ranges are whole
subtrees of the path tree where possible (block 0 is the most significant digit), so
every rank keeps the prefix sharing of its own subtrees.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def path_ranges(num_paths: int, world: int, subtree: int = 1) -> List[Tuple[int, int]]:
    """Split [0, num_paths) into `world` contiguous ranges whose boundaries are
    multiples of `subtree` (a subtree size of the path tree) when possible."""
    if world <= 0:
        raise ValueError("world must be positive")
    units = max(1, num_paths // subtree) if subtree > 0 else num_paths
    if num_paths % max(subtree, 1):
        units, subtree = num_paths, 1
    out = []
    for r in range(world):
        a = (units * r) // world * subtree
        b = (units * (r + 1)) // world * subtree
        out.append((a, min(b, num_paths)))
    out[-1] = (out[-1][0], num_paths)
    return out


def subtree_size(ranks: Sequence[int], world: int) -> int:
    """Largest subtree (product of the trailing Schmidt ranks) that still leaves at
    least one subtree per rank."""
    size, total = 1, 1
    for r in ranks:
        total *= r
    for r in reversed(ranks):
        if total // (size * r) < world:
            break
        size *= r
    return size


def allreduce_amplitudes(partial, group=None):
    """Sum complex128 partial amplitudes over the ranks (in place, returned).  With a
    gloo group a device tensor is reduced through a host copy."""
    import torch
    import torch.distributed as dist
    t = partial
    if partial.device.type != "cpu" and dist.get_backend(group) != "nccl":
        t = partial.cpu()
    dist.all_reduce(torch.view_as_real(t), op=dist.ReduceOp.SUM, group=group)
    if t is not partial:
        partial.copy_(t)
    return partial


def run_sharded(plan, bitstrings, rank: int, world: int, group=None):
    """This rank's share of the path sum of `plan` at `bitstrings`, reduced over ranks."""
    ranks = [int(x) for x in plan_ranks(plan)]
    lo, hi = path_ranges(int(plan.info["num_paths"]), world, subtree_size(ranks, world))[rank]
    out = plan.run(bitstrings, path_range=(lo, hi)) if hi > lo else None
    if out is None:
        import torch
        out = torch.zeros(bitstrings.numel(), dtype=torch.complex128, device=bitstrings.device)
    return allreduce_amplitudes(out, group)


def plan_ranks(plan):
    return [len(plan.sigma(k)) for k in range(int(plan.info["num_blocks"]))]
