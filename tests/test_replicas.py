"""Multi-process host logic on CPU (gloo, world size 2): the batch shards
cover every geometry exactly once with balanced cost, and the reported time
is the max over ranks."""
import os
import socket

import pytest

from paper_1609_04484_gb300.replicas import reduce_max, shard_by_cost


def test_shards_partition_and_balance():
    costs = [5.0, 1.0, 9.0, 3.0, 3.0, 7.0, 2.0, 8.0, 4.0, 6.0, 1.0]
    for world in (1, 2, 3, 4):
        parts = [shard_by_cost(costs, world, r) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT bound: the largest load is at most the mean plus the largest item
        assert max(loads) <= sum(costs) / world + max(costs)
    assert shard_by_cost([], 2, 1) == []
    with pytest.raises(ValueError):
        shard_by_cost(costs, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, costs, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard_by_cost(costs, world, rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        t = reduce_max(1.5 + rank)  # rank 1 is the slow one
        dist.barrier()
        out.put((rank, gathered, t))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_sharding_and_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    costs = [float((7 * i) % 11 + 1) for i in range(16)]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, t in res:
        assert sorted(i for part in gathered for i in part) == list(range(16))
        assert gathered[rank] == shard_by_cost(costs, 2, rank)
        assert t == 2.5
    assert reduce_max(3.0) == 3.0  # no process group in this process
