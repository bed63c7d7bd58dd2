"""Weak scaling of the bounding workload over ranks (one process per GPU).

The path shards without a data-path collective: rank r bounds its own batch of
nodes, drawn from the seeded generator with seed ``base + r``.  Only two scalars
cross ranks per measurement: each rank's elapsed time, reduced with MAX (the
job ends when its slowest rank ends), and its unit count (bounded children),
reduced with SUM.  The whole-job rate is total units / slowest time.
"""
from __future__ import annotations


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s node batch."""
    return base + rank


def node_range(count: int, rank: int, world: int) -> tuple[int, int]:
    """Half-open range [lo, hi) of the nodes of one batch that rank `rank` of
    `world` bounds when a single batch is split across ranks: contiguous,
    disjoint, covering [0, count), sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world or count < 0:
        raise ValueError("need 0 <= rank < world and count >= 0")
    return count * rank // world, count * (rank + 1) // world


def whole_job_rate(local_seconds: float, local_units: float, device=None):
    """(units per second over all ranks, slowest rank's seconds, total units).

    With torch.distributed initialised (any backend; `device` must suit it:
    a CUDA device for NCCL, the CPU for gloo) the two scalars are reduced
    across ranks; otherwise this rank's own figures are returned."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    seconds, units = t.item(), u.item()
    return (units / seconds if seconds > 0 else 0.0), seconds, units
