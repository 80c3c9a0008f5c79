"""Data-parallel training over ranks (one process per GPU).

Every rank keeps replicated parameters and a contiguous shard of each scene's
training pairs.  A step runs the fused training pass on the shard with the
loss normalised by the whole batch's pair count (`norm_pairs`), so the shard's
loss and gradients are its share of the batch's; one all-reduce (sum) over
the ranks then gives every rank the batch's loss and gradients, and every rank
applies the same Adam update (the loss scaler sees the same summed gradients
on every rank, so its skip / scale decisions agree).  The exchange is one
all-reduce of a flat buffer holding every gradient and the loss, through
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
    rank or without an initialised process group).  One collective per
    tensor: DataParallelStep packs a step's exchange into one tensor."""
    if not _distributed(group):
        return
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)


def _distributed(group=None):
    return dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1


def pack_losses(flat, losses):
    """Write the FP64 per-scene losses into the last 2 * len(losses) slots
    of the FP32 buffer flat as (hi, lo) pairs, hi = fp32(loss),
    lo = fp32(loss - hi): summed over ranks in FP32 and recombined in FP64
    they carry the batch loss to about FP32 rounding of the sum."""
    n = losses.numel()
    hi = losses.to(torch.float32)
    lo = (losses - hi.to(torch.float64)).to(torch.float32)
    tail = flat[flat.numel() - 2 * n:].view(n, 2)
    tail[:, 0] = hi
    tail[:, 1] = lo


def unpack_losses(flat, losses):
    """Inverse of pack_losses after the all-reduce: losses = hi + lo (FP64)."""
    n = losses.numel()
    tail = flat[flat.numel() - 2 * n:].view(n, 2).to(torch.float64)
    losses.copy_(tail[:, 0] + tail[:, 1])


def allreduce_flat(flat, losses, group=None):
    """The step's one exchange: pack the losses into the tail of the flat
    gradient buffer, all-reduce (sum) it once, unpack the losses."""
    if not _distributed(group):
        return
    pack_losses(flat, losses)
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    unpack_losses(flat, losses)


class DataParallelStep:
    """One data-parallel training step around a fused-mode TrainStep built on
    this rank's shard with `norm_pairs` = the batch's per-scene pair counts.
    The TrainStep's gradients are moved into one flat FP32 buffer with two
    slots per scene for its loss, so the step's exchange (every gradient and
    the loss) is a single all-reduce."""

    def __init__(self, step, group=None):
        if not step.fused or step.norm_pairs is None:
            raise ValueError("the shard's TrainStep needs the fused pass and norm_pairs")
        self.local = step
        self.group = group
        self.flat = step.use_flat_gradients(extra=2 * step.loss.numel())

    def gradients(self):
        return [g for pair in self.local.grads for g in pair]

    def fused_pass(self, stream=None):
        self.local.fused_pass(stream)

    def exchange(self, stream=None):
        ctx = torch.cuda.stream(stream) if stream is not None else _null()
        with ctx:
            allreduce_flat(self.flat, self.local.loss, self.group)

    def optimizer(self, stream=None):
        self.local.optimizer(stream)

    def step(self, stream=None):
        self.fused_pass(stream)
        self.exchange(stream)
        self.optimizer(stream)


class _null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False
