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

`backward_allreduce` overlaps that exchange with the last stage of the
backward instead: the projection backward (one thread per Gaussian, summing
its views) runs over contiguous ranges of Gaussians ("buckets"), and as soon
as a bucket's rows are final their all-reduce starts asynchronously (on
NCCL's stream, ordered after the work queued so far), while the next
bucket's projection backward runs.  The gradients are the same as with one
collective after the whole backward: each row is summed over the ranks once,
after every contribution to it.
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


def buckets(n: int, n_buckets: int) -> list:
    """Contiguous ranges of rows splitting [0, n) into at most n_buckets
    non-empty parts whose sizes differ by at most one, in order."""
    if n < 0 or n_buckets < 1:
        raise ValueError("buckets: need n >= 0 and n_buckets >= 1")
    k = min(n_buckets, n)
    return [range(b * n // k, (b + 1) * n // k) for b in range(k)]


def backward_allreduce(produce, grads, n: int, n_buckets: int = 4, group=None) -> None:
    """For each bucket of the rows [0, n) in order: `produce(first, count)`
    completes the gradient rows [first, first + count) of every array in
    `grads` (on the current stream), then the sum over the ranks of those
    rows starts asynchronously, one collective per array, overlapping the
    next bucket's `produce`.  Returns once every collective has been waited
    for (for NCCL: the current stream waits for them; on the CPU the call
    blocks).  With one rank only `produce` runs."""
    live = [g for g in grads if g is not None]
    multi = dist.is_initialized() and dist.get_world_size(group) > 1
    pending = []
    for b in buckets(n, n_buckets):
        produce(b.start, len(b))
        if multi:
            for g in live:
                pending.append(dist.all_reduce(g[b.start:b.stop], op=dist.ReduceOp.SUM,
                                               group=group, async_op=True))
    for w in pending:
        w.wait()


def project_allreduce(pipe, grads, n_buckets: int = 4, group=None, stream=None) -> None:
    """The bucketed projection backward of a SplatPipeline whose screen-space
    gradients are current (`pipe.backward_2d`, and the shading backward when
    shaded), with the all-reduce of each bucket's rows of `grads` = (mean_v,
    logscale_w, quat[, normal_beta, k_ads]) overlapping the next bucket."""
    import torch

    def produce(first, count):
        pipe.project_backward(grads[0], grads[1], grads[2], stream, first=first, count=count)
    if stream is None:
        backward_allreduce(produce, grads, pipe.n, n_buckets, group)
        return
    with torch.cuda.stream(stream):
        backward_allreduce(produce, grads, pipe.n, n_buckets, group)
