"""Data-parallel training host logic on CPU (two gloo ranks): view shards,
the one all-reduce of the flat gradient buffer against the oracle's
gradient summed over all views, the bucketed all-reduce overlapping the
projection backward (its order and its sums), the densification statistic,
and the parameter broadcast.  The library's own gradient kernels need a GPU:
here the oracle's per-shard gradients stand in for them."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2504_13339_gb300.parallel import view_shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_view_shards_partition_the_views():
    for n in range(0, 21):
        for world in range(1, 6):
            shards = [view_shard(n, r, world) for r in range(world)]
            assert [v for s in shards for v in s] == list(range(n))
            sizes = [len(s) for s in shards]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        view_shard(4, 2, 2)


def _scene():
    from paper_2504_13339_gb300 import scenes as S
    g = S.uniform_gaussians(60, 141, logscale_mean=-2.2)
    g.logscale_w[:, 3] = np.random.default_rng(142).uniform(0.4, 0.9, g.n)
    cams = S.orbit_cameras(5, 143, 24, 16)
    tfs = S.bump_tfs(1, 144)
    return g, cams, tfs


def _view_grads(g, cams, tfs, views):
    """The oracle's parameter gradients of a seeded per-view loss summed
    over `views` (mean_v, logscale_w, quat; float64)."""
    from oracle import veg_oracle as O
    sel = [cams[v] for v in views]
    if not sel:
        return [np.zeros((g.n, 4)) for _ in range(3)]
    proj, bins, fwd = O.render(sel, g, tfs, record=True)
    dout = np.stack([np.random.default_rng(150 + v).standard_normal(fwd["out"].shape[1:])
                     for v in views])
    g2 = O.composite_bwd(proj, sel, bins, tfs, (0, 0, 0), fwd, dout)
    return list(O.params_grad(sel, g, proj, g2))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2504_13339_gb300 import parallel
        from paper_2504_13339_gb300.train import DensityControl, TrainParams
        g, cams, tfs = _scene()
        P = TrainParams(g, device="cpu")
        flat = P.use_flat_gradients()
        assert all(gr.data_ptr() >= flat.data_ptr() for gr in P.grads if gr is not None)
        mine = _view_grads(g, cams, tfs, view_shard(len(cams), rank, world))
        for gr, part in zip(P.grads[:3], mine):
            gr.copy_(torch.as_tensor(part, dtype=torch.float32))
        parallel.allreduce_gradients(P)
        full = _view_grads(g, cams, tfs, range(len(cams)))
        errs = [float(np.abs(gr.numpy() - f).max() / max(np.abs(f).max(), 1e-30))
                for gr, f in zip(P.grads[:3], full)]
        # densification statistic: summed over the ranks
        dc = DensityControl(2.0, start=0, stop=10, every=5, device="cpu")
        dc.reset(g.n)
        dc.accum.fill_(float(rank + 1))
        dc.count.fill_(rank + 2)
        parallel.allreduce_density_stats(dc)
        stats = (float(dc.accum[0]), int(dc.count[-1]))
        # parameters: rank 0's everywhere after the broadcast
        if rank == 1:
            for t in P.raw[:3] + [P.mean_v]:
                t.add_(1.0)
        parallel.broadcast_parameters(P)
        P.step = 3
        parallel.sync_step(P)
        out[rank] = (errs, stats, float(P.raw[0].sum()), float(P.mean_v.sum()))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_all_reduce_the_view_gradients():
    from paper_2504_13339_gb300 import build
    build.build()
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(280)
        assert p.exitcode == 0
    for r in range(world):
        errs, stats, raw_sum, mean_sum = out[r]
        assert max(errs) <= 1e-5, errs  # float32 sums of float64 parts
        assert stats == (3.0, 5)
    assert out[0][2] == out[1][2] and out[0][3] == out[1][3]


def test_flat_gradients_survive_densification():
    """After the parameters adopt a densified storage, the gradient arrays
    are still consecutive [n][4] runs of the flat buffer (one collective
    covers them all) and restart at zero."""
    from paper_2504_13339_gb300 import build, scenes as S
    from paper_2504_13339_gb300.train import TrainParams
    build.build()
    g, lt = S.initial_model(40, S.blob_field(3, 145), 146, weight=0.3, lighting=True)
    P = TrainParams(g, lt, device="cpu")
    flat = P.use_flat_gradients()
    assert flat.numel() == 5 * 40 * 4
    for gr in P.grads:
        gr.fill_(1.0)
    for n2 in (55, 30, 90):
        rows = n2 + 7
        new = lambda: [torch.zeros(rows, 4) for _ in range(5)]
        store = (rows, new(), new(), new(), torch.zeros(rows, 4), torch.zeros(rows, 4))
        P.replace(n2, store)
        assert P.flat_grads.numel() == 5 * n2 * 4
        base = P.flat_grads.data_ptr()
        for a, gr in enumerate(P.grads):
            assert gr.shape == (n2, 4) and gr.data_ptr() == base + a * n2 * 16
            assert not gr.any()
        P.flat_grads.fill_(2.0)
        assert all(bool((gr == 2.0).all()) for gr in P.grads)


def _rank_steps(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2504_13339_gb300 import parallel

        class P:  # only what sync_step reads
            raw = [torch.zeros(1)]
            step = 5 + rank  # rank 1 took one extra step
        try:
            parallel.sync_step(P)
            out[rank] = "no error"
        except RuntimeError as e:
            out[rank] = str(e)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_ranks_at_different_steps_are_reported_on_every_rank():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_steps, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(100)
        assert p.exitcode == 0
    for r in range(world):
        assert "different steps (5 .. 6)" in out[r]


def test_buckets_partition_the_rows():
    from paper_2504_13339_gb300.parallel import buckets
    for n in range(0, 40):
        for k in range(1, 9):
            bs = buckets(n, k)
            assert [i for b in bs for i in b] == list(range(n))
            assert all(len(b) > 0 for b in bs) and len(bs) == min(n, k)
            if bs:
                assert max(map(len, bs)) - min(map(len, bs)) <= 1
    with pytest.raises(ValueError):
        buckets(5, 0)


def _rank_buckets(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2504_13339_gb300 import parallel
        from paper_2504_13339_gb300.train import TrainParams
        g, cams, tfs = _scene()
        P = TrainParams(g, device="cpu")
        P.use_flat_gradients()
        grads = P.grads[:3]
        mine = [torch.as_tensor(a, dtype=torch.float32)
                for a in _view_grads(g, cams, tfs, view_shard(len(cams), rank, world))]
        log, produced = [], set()
        bases = [(gr.data_ptr(), gr.data_ptr() + gr.numel() * 4) for gr in grads]

        def produce(first, count):
            log.append(("p", first, count))
            for gr, part in zip(grads, mine):
                gr[first:first + count] = part[first:first + count]
            produced.update(range(first, first + count))

        real = dist.all_reduce

        def logged(t, *a, **kw):
            arr = next(i for i, (lo, hi) in enumerate(bases) if lo <= t.data_ptr() < hi)
            row = (t.data_ptr() - bases[arr][0]) // 16
            rows = range(row, row + t.shape[0])
            log.append(("r", arr, row, t.shape[0], set(rows) <= produced, kw.get("async_op")))
            return real(t, *a, **kw)
        dist.all_reduce = logged
        try:
            parallel.backward_allreduce(produce, grads, g.n, n_buckets=4)
        finally:
            dist.all_reduce = real
        full = _view_grads(g, cams, tfs, range(len(cams)))
        errs = [float(np.abs(gr.numpy() - f).max() / max(np.abs(f).max(), 1e-30))
                for gr, f in zip(grads, full)]
        out[rank] = (log, errs)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_bucketed_allreduce_follows_each_bucket_and_sums_the_views():
    """Each bucket's rows are all-reduced (asynchronously, one collective per
    gradient array) right after that bucket is produced and before the next
    bucket is, never before its rows are final; the summed gradients equal
    the oracle's gradient over all views."""
    from paper_2504_13339_gb300 import build
    build.build()
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_buckets, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(280)
        assert p.exitcode == 0
    n = _scene()[0].n
    from paper_2504_13339_gb300.parallel import buckets
    want = []
    for b in buckets(n, 4):
        want.append(("p", b.start, len(b)))
        want += [("r", a, b.start, len(b), True, True) for a in range(3)]
    for r in range(world):
        log, errs = out[r]
        assert log == want
        assert max(errs) <= 1e-5, errs
