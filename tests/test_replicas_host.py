"""Host logic of the multi-GPU modes, run as two gloo processes on the CPU:
the replicated benchmark takes the slowest rank's time and counts every
rank's work; a served stream splits into disjoint per-GPU shards that cover
it and balance the work."""
import os
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1911_08158_gb300 import workloads as wl
    from paper_1911_08158_gb300.serve import request_dofs, shard_requests
    t = bench.max_over_ranks(1.0 + rank, world)
    value = bench.replica_value(100.0, world, t)
    reqs = wl.serving_requests(count=60, rate=50.0, seed=4, lo=8, hi=40, max_steps=50)
    mine = shard_requests(reqs, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, [r.rid for r in mine])
    work = sum(request_dofs(r) * r.steps for r in mine)
    works = [None] * world
    dist.all_gather_object(works, work)
    out[rank] = (t, value, gathered, works)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_and_shards_with_two_gloo_ranks():
    world = 2
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, value, gathered, works = res[rank]
        assert t == 2.0                       # the slowest rank
        assert value == 100.0 * world / 2.0   # all ranks' units over that time
        ids = [i for shard in gathered for i in shard]
        assert sorted(ids) == list(range(60)) and len(set(ids)) == 60
        assert max(works) <= 1.6 * min(works)  # greedy balance
