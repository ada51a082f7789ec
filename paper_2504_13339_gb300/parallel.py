"""Data-parallel training over views, one process per GPU.

The views of a training step are independent until the per-Gaussian
gradients are summed (Sec. 4.2: the loss is a sum over the training images),
so a step shards its views across the ranks: every rank holds the whole
model, renders and differentiates its own contiguous share of the views,
and one all-reduce (sum) of the gradient arrays gives every rank the
gradient of the whole batch.  Every rank then takes the same Adam step on
the same parameters, so the replicas stay identical without exchanging
parameters.  With density control the positional-gradient statistic is a
sum over views too: it is all-reduced before the clone/split/prune
decisions, which every rank then takes identically (same statistic, same
seeded draws).

The collective is torch.distributed's all_reduce on one flat buffer (NCCL
between GPUs, gloo on the CPU); the gradient arrays of `TrainParams` are
views into that buffer (`TrainParams.use_flat_gradients`), so a step needs
one collective and no packing.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def view_shard(n_views: int, rank: int, world: int) -> range:
    """The contiguous views of `rank` among `world` ranks (sizes differ by at
    most one; every view belongs to exactly one rank)."""
    if world < 1 or not 0 <= rank < world or n_views < 0:
        raise ValueError("view_shard: need 0 <= rank < world and n_views >= 0")
    return range(rank * n_views // world, (rank + 1) * n_views // world)


def allreduce_gradients(params, group=None) -> None:
    """Sums the gradient arrays of `params` (a TrainParams using flat
    gradients) over the ranks of `group`, in place."""
    flat = params.flat_grads
    if flat is None:
        raise ValueError("allreduce_gradients: call params.use_flat_gradients() first")
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)


def allreduce_density_stats(density, group=None) -> None:
    """Sums the densification statistic (accumulated gradient norms and
    counts) over the ranks, so that every rank clones, splits and prunes the
    same Gaussians."""
    if density.accum is None:
        return
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(density.accum, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(density.count, op=dist.ReduceOp.SUM, group=group)


def broadcast_parameters(params, src=0, group=None) -> None:
    """Makes every rank's parameters and Adam state those of `src` (once, at
    the start of a data-parallel run)."""
    if not (dist.is_initialized() and dist.get_world_size(group) > 1):
        return
    for t in params.raw + params.m + params.v + [params.mean_v, params.logscale_w]:
        if t is not None:
            dist.broadcast(t, src=src, group=group)


def sync_step(params, group=None) -> None:
    """Checks that every rank is at the same Adam step (cheap guard against a
    rank that skipped an iteration)."""
    if not (dist.is_initialized() and dist.get_world_size(group) > 1):
        return
    dev = params.raw[0].device
    t = torch.tensor([params.step], dtype=torch.int64, device=dev)
    lo, hi = t.clone(), t.clone()
    dist.all_reduce(lo, op=dist.ReduceOp.MIN, group=group)
    dist.all_reduce(hi, op=dist.ReduceOp.MAX, group=group)
    if int(lo) != int(hi):
        raise RuntimeError(f"ranks are at different steps ({int(lo)} .. {int(hi)})")
