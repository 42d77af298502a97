"""Multi-process forms of the search (one process per GPU).

Two layouts:
* replicas -- every rank holds the whole database and searches its own
  query stream; the only exchange is the benchmark's max-over-ranks time and
  the sum of queries (``aggregate``).
* row shards -- rank r holds rows [r0, r1) (``shard_bounds``); every rank
  searches the same queries against its shard, the per-shard (Delta, id)
  lists are all-gathered and merged into the global top-k
  (``gather_and_merge``; on GPUs the merge is libevp's evp_merge_topk).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_bounds(ns: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous row range of `rank` when ns rows are split over `world` ranks."""
    base, extra = divmod(ns, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def aggregate(units_local: float, ms_local: float, device=None) -> tuple[float, float]:
    """(units summed over ranks, max elapsed ms over ranks)."""
    if not (dist.is_available() and dist.is_initialized()):
        return float(units_local), float(ms_local)
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()), float(t.item())


def gather_and_merge(ids_local: torch.Tensor, dist_local: torch.Tensor, k: int, merge,
                     row_offset: int = 0):
    """All-gather per-shard results ([nq, k] ids local to the shard, int32
    Delta) and merge them into the global top-k with `merge(ids[P, nq, k],
    dist[P, nq, k], k)`.  Shard-local ids are shifted by `row_offset`; -1
    (no candidate) stays -1."""
    ids_g = torch.where(ids_local >= 0, ids_local + int(row_offset), ids_local)
    if dist.is_available() and dist.is_initialized():
        world = dist.get_world_size()
        all_ids = [torch.empty_like(ids_g) for _ in range(world)]
        all_dist = [torch.empty_like(dist_local) for _ in range(world)]
        dist.all_gather(all_ids, ids_g.contiguous())
        dist.all_gather(all_dist, dist_local.contiguous())
        ids_s, dist_s = torch.stack(all_ids), torch.stack(all_dist)
    else:
        ids_s, dist_s = ids_g[None], dist_local[None]
    return merge(ids_s.contiguous(), dist_s.contiguous(), k)
