"""Host logic of one solve split over ranks by views (CPU, gloo, world size 2):
the view ranges partition the views, and the all-reduce of the nine per-pixel
channels gives every rank the sum over all views."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1801_06263_gb300 import split


@pytest.mark.parametrize("n_views,world", [(512, 1), (512, 2), (90, 4), (7, 7), (1000, 3), (5, 2)])
def test_view_ranges_partition_the_views(n_views, world):
    ranges = [split.view_range(n_views, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n_views
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0
    sizes = [v1 - v0 for v0, v1 in ranges]
    assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1


def test_view_range_rejects_more_ranks_than_views():
    with pytest.raises(ValueError):
        split.view_range(3, 0, 4)
    with pytest.raises(ValueError):
        split.view_range(8, 2, 2)


def _per_view_channels(v0, v1, P):
    # a stand-in for the back-projected channels of views [v0, v1): exact small integers
    v = torch.arange(v0, v1, dtype=torch.float32)
    k = torch.arange(P, dtype=torch.float32)
    return torch.stack([((v[:, None] + c) % 7 + k[None, :] % 3).sum(0) for c in range(9)])


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n_views, P = 37, 50
    v0, v1 = split.view_range(n_views, rank, world)
    chan = _per_view_channels(v0, v1, P)
    split.allreduce_channels(chan)
    out[rank] = (v0, v1, chan.numpy().tolist())
    dist.destroy_process_group()


def test_allreduce_gives_every_rank_the_full_sum():
    port = 29600 + os.getpid() % 1000
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        full = _per_view_channels(0, 37, 50)
        assert out[0][1] == out[1][0]
        for rank in range(2):
            assert torch.equal(torch.tensor(out[rank][2]), full)
