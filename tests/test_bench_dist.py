"""The benchmark's multi-rank aggregation on CPU (gloo, world size 2): each GPU
runs independent solves, the whole-job rate is all ranks' units over the
slowest rank's time, and only rank 0 prints."""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, _ = bench._dist()
    assert (ws, r) == (world, rank)
    bench._barrier(ws)
    rate, t = bench.whole_job_rate(ws, 100, 2.0 + rank)    # rank 1 is the slow one: 3 s
    out[rank] = (rate, t)
    dist.destroy_process_group()


def test_whole_job_rate_uses_slowest_rank():
    port = 29500 + os.getpid() % 1000
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        for rank in range(2):
            rate, t = out[rank]
            assert t == pytest.approx(3.0)
            assert rate == pytest.approx(2 * 100 / 3.0)
