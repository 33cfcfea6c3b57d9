"""The replica aggregation of bench.py under two gloo ranks on CPU: the job's
throughput is the cells of all ranks over the slowest rank's time."""
import os

import pytest
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.aggregate(elapsed_ms=100.0 * (rank + 1), cells_per_rank=1_000_000, steps=10, dist=dist)
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        ms, value = out[r]
        assert ms == pytest.approx(20.0)                      # slowest rank: 200 ms over 10 steps
        assert value == pytest.approx(2 * 1_000_000 / 0.020 / 1e6)
