"""Sharding of independent instances across ranks, checked with world_size-2 gloo process groups
on the CPU: every instance is owned by exactly one rank, all ranks agree, loads are balanced."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2406_04177_gb300.shard import rank_loads, shard_instances


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, sizes, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard_instances(sizes, world, rank)
    everyone = [None] * world
    dist.all_gather_object(everyone, mine)
    # each rank's view of every rank's share must agree with what that rank computed itself
    agree = all(everyone[r] == shard_instances(sizes, world, r) for r in range(world))
    dist.destroy_process_group()
    q.put((rank, mine, everyone, agree))


@pytest.mark.parametrize("world", [2])
def test_gloo_ranks_partition_instances(world):
    sizes = [5000, 120, 88000, 4300, 4300, 17, 64000, 900, 0, 33000, 12000]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, sizes, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    results.sort()
    assert all(r[3] for r in results)
    owned = sorted(i for r in results for i in r[1])
    assert owned == list(range(len(sizes)))
    loads = rank_loads(sizes, world)
    assert max(loads) - min(loads) <= max(sizes)


def test_single_rank_owns_all():
    assert shard_instances([3, 1, 2], 1, 0) == [0, 1, 2]
    with pytest.raises(ValueError):
        shard_instances([1], 2, 2)
