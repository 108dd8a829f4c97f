"""Multi-GPU layout of the signature path: independent shards, no data-path exchange.

Polygons are independent (Definition 2 hashes one polygon at a time), so N ranks each
sign, index and query their own shard of the same size (weak scaling).  The only
communication is timing: a barrier on both sides of the timed region and the maximum
step time over ranks.  The launcher is torchrun (one process per GPU); rank 0 reports.
"""
from __future__ import annotations

import dataclasses
import os


def env():
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_workload(w, rank: int):
    """Rank r signs its own synthetic shard: same sizes, generator seed offset by 1000 r."""
    if rank == 0:
        return w
    return dataclasses.replace(w, gen_seed=w.gen_seed + 1000 * rank,
                               query_seed=w.query_seed + 1000 * rank)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar (the step time) over the process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, step_seconds: float) -> float:
    """Whole-job throughput: units all ranks processed per second of the slowest rank."""
    return units_per_rank * world / step_seconds
