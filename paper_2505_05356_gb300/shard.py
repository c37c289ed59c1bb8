"""Frames of a batch split over processes (one GPU each).

Frames are independent through the whole forward and backward; only the
parameter gradients sum over frames.  So a batch shards by contiguous frame
ranges with no exchange on the render path, and a sharded *fit* needs one
collective per iteration: the sum of the parameter gradients over the shards
before the Adam step, which then runs identically on every process.
:func:`allreduce_sum_` is that step (one flattened buffer, one all-reduce;
NCCL between GPUs, gloo between CPU processes); `fit.FitLoop(grad_hook=...)`
calls it between the backward and the update.
"""
from __future__ import annotations

from typing import Iterable, Optional, Tuple

import torch


def frame_range(n_frames: int, world: int, rank: int) -> Tuple[int, int]:
    """[start, stop) of rank's frames: contiguous, sizes differing by at most
    one, the larger shards first; empty when world > n_frames for the last
    ranks."""
    if n_frames < 0 or world < 1 or not 0 <= rank < world:
        raise ValueError("bad shard request (%d frames, world %d, rank %d)"
                         % (n_frames, world, rank))
    base, extra = divmod(n_frames, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def allreduce_sum_(tensors: Iterable[torch.Tensor], group: Optional[object] = None):
    """Sum each tensor over the processes of `group` in place (one all-reduce
    of one flattened buffer).  All tensors share a device and dtype."""
    import torch.distributed as dist

    ts = [t for t in tensors if t is not None and t.numel() > 0]
    if not ts:
        return
    flat = torch.cat([t.reshape(-1) for t in ts])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    at = 0
    for t in ts:
        n = t.numel()
        t.copy_(flat[at:at + n].view_as(t))
        at += n
