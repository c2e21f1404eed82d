"""Host-side logic for runs over several GPUs (one process per GPU).

The method has no exchange step between independent samples, so an ensemble
is sharded by sample with no data-path collective; a single coupled domain
runs as independent replicas.  The only collectives are for timing and
reporting (max of the per-rank times, sums of the per-rank work).
"""
from __future__ import annotations

from typing import List, Sequence


def shard_samples(sites: Sequence[int], rank: int, world: int) -> List[int]:
    """Indices of the samples rank `rank` owns: greedy largest-first
    assignment to the least-loaded rank (deterministic, balanced in sites)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank / world")
    order = sorted(range(len(sites)), key=lambda i: (-sites[i], i))
    load = [0] * world
    owner = [0] * len(sites)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += sites[i]
    return [i for i in range(len(sites)) if owner[i] == rank]


def max_over_ranks(x: float, device="cpu") -> float:
    """Maximum of a per-rank scalar (identity without torch.distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device="cpu") -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units_per_rank: float, seconds_per_rank: float, device="cpu") -> float:
    """Whole-job throughput: sum of every rank's units over the slowest rank's time."""
    units = sum_over_ranks(units_per_rank, device)
    t = max_over_ranks(seconds_per_rank, device)
    return units / t if t > 0 else float("inf")
