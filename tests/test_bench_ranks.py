"""The multi-GPU path of bench.py runs independent replicas, one per rank,
with no data-path collective; the whole-job figures sum the ranks' flips and
take the slowest rank's time.  Checked here with two gloo ranks on the CPU."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out = bench.aggregate_ranks(1000 * (rank + 1), 10.0 + rank, 7 * (rank + 1), 1.5 + 0.5 * rank, dist)
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        flips, ms, ef, et = res[r]
        assert flips == 3000 and ms == 11.0 and ef == 21 and et == 2.0


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(5, 2.0, 3, 1.0, None) == (5, 2.0, 3, 1.0)
