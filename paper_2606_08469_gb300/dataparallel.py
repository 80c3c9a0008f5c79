"""Data-parallel training over ranks (one process per GPU).

Every rank keeps replicated parameters and a contiguous shard of each scene's
training pairs.  A step runs the fused training pass on the shard with the
loss normalised by the whole batch's pair count (`norm_pairs`), so the shard's
loss and gradients are its share of the batch's; one all-reduce (sum) over
the ranks then gives every rank the batch's loss and gradients, and every rank
applies the same Adam update (the loss scaler sees the same summed gradients
on every rank, so its skip / scale decisions agree).  The all-reduce is
`torch.distributed` (NCCL between GPUs, gloo on CPU).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_range(n, rank, world):
    """Contiguous, balanced shard [begin, end) of n items for a rank."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside [0, {world})")
    base, extra = divmod(int(n), int(world))
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def allreduce_sum(tensors, group=None):
    """Sum each tensor over the ranks of the group, in place (no-op on one
    rank or without an initialised process group)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)


class DataParallelStep:
    """One data-parallel training step around a fused-mode TrainStep built on
    this rank's shard with `norm_pairs` = the batch's per-scene pair counts."""

    def __init__(self, step, group=None):
        if not step.fused or step.norm_pairs is None:
            raise ValueError("the shard's TrainStep needs the fused pass and norm_pairs")
        self.local = step
        self.group = group

    def gradients(self):
        return [g for pair in self.local.grads for g in pair]

    def step(self, stream=None):
        s = self.local
        s.fused_pass(stream)
        ctx = torch.cuda.stream(stream) if stream is not None else _null()
        with ctx:
            allreduce_sum(self.gradients() + [s.loss], self.group)
        s.optimizer(stream)


class _null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False
