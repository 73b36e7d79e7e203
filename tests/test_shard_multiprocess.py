"""Multi-rank host logic on the CPU (gloo, world size 2): each rank takes its
cost-balanced shard of the batched workload's LIZs; the shards are disjoint,
cover every LIZ, and their n^3 costs are balanced.  No GPU is used."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2308_16317_gb300 import shard
    from paper_2308_16317_gb300 import workload as wl
    w = wl.batched_supercell(n_sites=64)
    orders = [w.n_of(l) for l in w.lizs]
    mine = shard.balanced_shards(orders, world)[rank]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    import torch
    t = torch.tensor([shard.shard_cost(orders, mine)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((gathered, float(t.item()), orders))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_are_disjoint_complete_and_balanced():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, max_cost, orders = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    a, b = set(gathered[0]), set(gathered[1])
    assert not (a & b)
    assert a | b == set(range(len(orders)))
    total = sum(float(n) ** 3 for n in orders)
    assert max_cost <= 0.5 * total * 1.05


def test_single_rank_shard_is_everything():
    from paper_2308_16317_gb300 import shard
    orders = [688, 2160, 1264, 880]
    assert shard.balanced_shards(orders, 1) == [[0, 1, 2, 3]]
    assert sorted(sum(shard.balanced_shards(orders, 3), [])) == [0, 1, 2, 3]
