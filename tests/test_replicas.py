"""Host-side logic of multi-GPU runs (replicas and sharded batches), on the
CPU: balanced disjoint shards, and the collectives bench.py uses (maximum
over ranks, gather to rank 0) in a world of 2 gloo processes."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1601_04641_gb300 import inputs, replicas


def test_shards_cover_every_instance_once_and_balance():
    sizes = [p.sites for p in inputs.batch_problems(64, seed=0)]
    for world in (1, 2, 3, 4, 8):
        shares = [replicas.shard_by_sites(sizes, r, world) for r in range(world)]
        flat = sorted(i for s in shares for i in s)
        assert flat == list(range(64))
        loads = [sum(sizes[i] for i in s) for s in shares]
        assert max(loads) - min(loads) <= max(sizes)
    with pytest.raises(ValueError):
        replicas.shard_by_sites(sizes, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = [p.sites for p in inputs.batch_problems(16, seed=4)]
        mine = replicas.shard_by_sites(sizes, rank, world)
        slowest = replicas.max_over_ranks(1.5 + rank, dist)        # per-rank "elapsed"
        gathered = replicas.gather_to_rank0({"rank": rank, "mine": mine}, dist)
        out.put((rank, mine, slowest, gathered))
    finally:
        dist.destroy_process_group()


def test_collectives_with_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = {}
    for _ in range(world):
        rank, mine, slowest, gathered = q.get(timeout=120)
        results[rank] = (mine, slowest, gathered)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert results[0][1] == results[1][1] == 2.5                   # the maximum over ranks
    assert sorted(results[0][0] + results[1][0]) == list(range(16))  # disjoint shares
    assert results[1][2] is None
    assert [g["rank"] for g in results[0][2]] == [0, 1]
    assert [g["mine"] for g in results[0][2]] == [results[0][0], results[1][0]]
    assert replicas.max_over_ranks(3.0) == 3.0 and replicas.gather_to_rank0(7) == [7]
