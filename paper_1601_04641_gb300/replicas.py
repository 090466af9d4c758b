"""Host-side logic of runs on several GPUs of one node, one process per GPU.

A single condensate does not shard here (every run has one grid per GPU), so
several GPUs run independent work: replicas of the same workload, or disjoint
shares of a batch of independent condensates.  Nothing in the data path is
exchanged; the only collectives are the timing barrier, a maximum over ranks
and the gather of per-rank results to rank 0 (torch.distributed, any backend).
"""
from __future__ import annotations


def shard_by_sites(sizes, rank, world):
    """Indices of the items (given by their site counts) that `rank` of
    `world` takes: largest first, each to the rank with the fewest sites so
    far (ties to the lower rank), so the shares are disjoint, cover every
    item and differ by at most the largest item.  Deterministic."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    load = [0] * world
    mine = []
    for i in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += sizes[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def max_over_ranks(value, dist=None, device="cpu"):
    """The maximum of a float over all ranks (the value itself without a
    process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_to_rank0(obj, dist=None):
    """Every rank's `obj`, in rank order, on rank 0 (None on other ranks);
    [obj] without a process group."""
    if dist is None:
        return [obj]
    out = [None] * dist.get_world_size() if dist.get_rank() == 0 else None
    dist.gather_object(obj, out, dst=0)
    return out
