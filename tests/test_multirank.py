"""The multi-GPU form is independent replicas (queries shard with no data
exchange): each rank runs its own batch; the benchmark reports the units of
all ranks over the slowest rank's time.  This checks that host logic with
world size 2 over gloo on the CPU."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    secs = [2.0, 3.0][rank]          # rank 1 is the slower replica
    units = [256 * 10, 256 * 10][rank]
    tmax, utot, val = bench.aggregate(secs, units, dist)
    ws, rk, _ = bench.dist_env()
    q.put((rank, tmax, utot, val, ws, rk))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, utot, val, ws, rk in res:
        assert rk == rank and ws == 2
        assert tmax == 3.0 and utot == 5120.0
        assert val == pytest.approx(5120.0 / 3.0)


def test_single_rank_aggregate_without_dist():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(2.0, 512, None) == (2.0, 512.0, 256.0)
