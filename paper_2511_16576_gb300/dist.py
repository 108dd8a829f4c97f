"""Multi-GPU layout of the signature path: polygon shards, one exchange for the search.

Polygons are independent (Definition 2 hashes one polygon at a time), so N ranks each
sign and index their own shard of the database (weak scaling: same shard size per
rank) with no data-path collective.  The nearest-neighbour search over the whole
database (Definition 1, refined by exact Jaccard as in Sec. 5.2) has one real exchange:

1. all-gather of the query batch -- every rank's query signatures (Q_r x K uint32) and
   query vertices (the exact refinement needs the query's geometry on every shard);
2. on every rank, the local search of all gathered queries against its own shard
   (bucket join, agreement, refinement), giving per query its shard's top-k as
   (exact J, global polygon id);
3. all-gather of those per-shard top-k lists and, on each query's own rank, the merge
   by (J desc, global id asc) -- the order of a single search over the union.

Every collective is a plain all_gather of padded, equal-size tensors (NCCL on GPUs,
gloo in the CPU tests); no peer memory and no multicast.  The launcher is torchrun
(one process per GPU); rank 0 reports.
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


def shard_offsets(n_local: int, device=None):
    """Global id of every rank's first polygon (ranks' shards concatenated in rank order):
    int64 tensor [world + 1]."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_initialized() else 1
    sizes = _all_gather_rows(torch.tensor([n_local], dtype=torch.int64, device=device))
    out = torch.zeros(world + 1, dtype=torch.int64, device=device)
    out[1:] = torch.cumsum(torch.cat(sizes), 0)
    return out


def _all_gather_rows(t):
    """All-gather of a tensor whose first dimension differs between ranks: pads to the
    longest, gathers, and trims each rank's part.  Returns the list of parts."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return [t]
    world = dist.get_world_size()
    n = torch.tensor([t.shape[0]], dtype=torch.int64, device=t.device)
    ns = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(ns, n)
    ns = [int(x.item()) for x in ns]
    longest = max(max(ns), 1)
    pad = torch.zeros((longest,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
    pad[:t.shape[0]] = t
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return [p[:m] for p, m in zip(parts, ns)]


@dataclasses.dataclass
class QueryBatch:
    """A batch of queries: signatures uint32 [Q, K] (in int32; None when every shard signs
    the gathered queries itself), vertices int32 [V, 2], offsets int64 [Q + 1]."""
    sig: "object"
    xy: "object"
    offsets: "object"

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0]) - 1


def gather_queries(qb: QueryBatch):
    """Step 1: every rank's query batch, concatenated in rank order, and the range of
    this rank's own queries in it."""
    import torch
    import torch.distributed as dist
    sigs = _all_gather_rows(qb.sig) if qb.sig is not None else None
    xys = _all_gather_rows(qb.xy)
    offs = _all_gather_rows(qb.offsets[1:] - qb.offsets[0])   # per-rank ends, from 0
    rank = dist.get_rank() if dist.is_initialized() else 0
    out_off = [torch.zeros(1, dtype=torch.int64, device=qb.offsets.device)]
    base, q0, mine = 0, 0, (0, 0)
    for r, (o, x) in enumerate(zip(offs, xys)):
        out_off.append(o + base)
        if r == rank:
            mine = (q0, q0 + o.shape[0])
        base += x.shape[0]
        q0 += o.shape[0]
    return QueryBatch(torch.cat(sigs) if sigs is not None else None, torch.cat(xys),
                      torch.cat(out_off)), mine


def merge_topk(j_parts, id_parts, k: int):
    """Per query, the k best of the shards' lists by (J desc, global id asc).

    j_parts / id_parts: lists (one per shard) of [Q, k_s] tensors (float64 J, int64 global
    ids); empty slots carry id -1 and are dropped.  Returns ([Q, k] ids with -1 padding,
    [Q, k] J with -1 padding)."""
    import torch
    j = torch.cat(j_parts, 1)
    ids = torch.cat(id_parts, 1)
    empty = ids < 0
    j = torch.where(empty, torch.full_like(j, -1.0), j)
    big = torch.iinfo(torch.int64).max
    key_id = torch.where(empty, torch.full_like(ids, big), ids)
    # (J desc, id asc): stable sort by id, then stable sort by -J
    o1 = torch.sort(key_id, dim=1, stable=True).indices
    j1, id1 = torch.gather(j, 1, o1), torch.gather(ids, 1, o1)
    o2 = torch.sort(-j1, dim=1, stable=True).indices
    j2, id2 = torch.gather(j1, 1, o2)[:, :k], torch.gather(id1, 1, o2)[:, :k]
    id2 = torch.where(j2 < 0, torch.full_like(id2, -1), id2)
    if id2.shape[1] < k:
        pad = k - id2.shape[1]
        id2 = torch.cat([id2, torch.full((id2.shape[0], pad), -1, dtype=id2.dtype,
                                         device=id2.device)], 1)
        j2 = torch.cat([j2, torch.full((j2.shape[0], pad), -1.0, dtype=j2.dtype,
                                       device=j2.device)], 1)
    return id2, j2


def global_search(local_search, qb: QueryBatch, shard_base: int, k: int = 10):
    """Steps 1-3 for this rank's query batch.

    local_search(all_queries: QueryBatch, k) -> (ids [Q_all, k] local ids or -1,
    J [Q_all, k] float64) searches this rank's shard for every gathered query;
    shard_base is the global id of this rank's first polygon.  Returns the merged
    (global ids, J) of this rank's own queries, [Q_r, k] each."""
    import torch
    allq, (q0, q1) = gather_queries(qb)
    ids, j = local_search(allq, k)
    gids = torch.where(ids >= 0, ids.to(torch.int64) + shard_base, torch.full_like(ids, -1,
                                                                                 dtype=torch.int64))
    j_parts = _all_gather_rows(j.to(torch.float64).contiguous())
    id_parts = _all_gather_rows(gids.contiguous())
    return merge_topk([p[q0:q1] for p in j_parts], [p[q0:q1] for p in id_parts], k)
