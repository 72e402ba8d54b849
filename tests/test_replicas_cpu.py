"""The multi-GPU form of the bench workloads is replicas: each rank runs its own
share of independent problems, and the job's time is the slowest rank's.
These tests run that host logic with gloo ranks on CPU (world size 2)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2406_16796_gb300 import workloads as W


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    scan = W.shard(W.scan_instances(), rank, world)
    reqs = W.shard(W.serve_requests(count=50), rank, world)
    slowest = bench.max_over_ranks(1.5 + rank, world, device="cpu")
    out.put((rank, [(i.nx, i.steps) for i in scan], [r.arrival for r in reqs], slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_ranks_split_the_problems_disjointly_and_time_the_slowest():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict((x[0], x[1:]) for x in (q.get(timeout=120) for _ in range(world)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    every = [(i.nx, i.steps) for i in W.scan_instances()]
    mine = [got[r][0] for r in range(world)]
    assert sorted(mine[0] + mine[1]) == sorted(every)
    assert len(mine[0]) == len(mine[1]) == len(every) // 2
    arrivals = [got[r][1] for r in range(world)]
    assert sorted(arrivals[0] + arrivals[1]) == sorted(r.arrival for r in W.serve_requests(count=50))
    assert got[0][2] == got[1][2] == 2.5  # every rank reports the slowest rank's time



def test_shard_rejects_bad_ranks():
    with pytest.raises(ValueError):
        W.shard([1, 2, 3], 2, 2)
    assert W.shard([1, 2, 3, 4, 5], 1, 2) == [2, 4]
