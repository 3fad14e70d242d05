"""One solve shared by several ranks (one GPU each): the views are split into
contiguous ranges, one per rank.  Each MOCCA iteration, every rank runs the
ray side for its own views (osscir_mocca_partial: forward projection, counts
model, curvature, dual step and the back-projection of the nine per-pixel
channels), the channels are summed over the ranks by one all-reduce of 9 P
floats, and every rank takes the same primal step (osscir_mocca_apply), so
all ranks hold the same maps.  The forward and back-projections that Sec. 1
and 2 name as the cost are sums over rays, which is what makes the split exact
up to the order of the floating-point additions.

This module only orchestrates the library calls and the collective; all
arithmetic of the method runs in the CUDA library.
"""
from __future__ import annotations

from . import _lib


def view_range(n_views: int, rank: int, world: int) -> tuple[int, int]:
    """The contiguous views [v0, v1) of rank `rank` of `world`: sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or n_views < world:
        raise ValueError("need 0 <= rank < world <= n_views")
    base, extra = divmod(n_views, world)
    v0 = rank * base + min(rank, extra)
    return v0, v0 + base + (1 if rank < extra else 0)


def allreduce_channels(chan, group=None):
    """Sum chan ([9, P]) over the ranks in place.  NCCL reduces device tensors
    directly; other backends (gloo) go through a host copy."""
    import torch.distributed as dist
    if dist.get_backend(group) == "nccl" or not chan.is_cuda:
        dist.all_reduce(chan, group=group)
        return chan
    host = chan.cpu()
    dist.all_reduce(host, group=group)
    chan.copy_(host)
    return chan


class SplitSolve:
    """MOCCA iterations of `recon` (a Reconstructor of the shared problem, in the
    same state on every rank) with the views split over the process group."""

    def __init__(self, recon, rank: int, world: int, group=None):
        import torch
        self.recon, self.group = recon, group
        self.v0, self.v1 = view_range(recon.geom.n_views, rank, world)
        self.chan = torch.zeros((9, recon.n_pixels), dtype=torch.float32, device="cuda")

    def step(self, n_iters: int, stream=None):
        for _ in range(int(n_iters)):
            _lib.osscir_mocca_partial(self.recon.handle, self.v0, self.v1, self.chan, stream)
            allreduce_channels(self.chan, self.group)
            _lib.osscir_mocca_apply(self.recon.handle, self.chan, stream)
