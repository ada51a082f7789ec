"""Serving loop: every result is the same rendered alone and in the mix, and
a per-view-TF batch equals the matching single renders."""
import numpy as np
import pytest
import torch

from paper_2504_13339_gb300 import _lib, scenes as S
from paper_2504_13339_gb300.serve import (Request, RenderServer, SlotLimits, fifo_serve,
                                          latency_stats, poisson_requests)


def test_poisson_requests_are_seeded_and_in_range():
    models = {"a": None, "b": None}
    r1 = poisson_requests(models, 5, rate=50.0, duration=2.0, seed=3)
    r2 = poisson_requests(models, 5, rate=50.0, duration=2.0, seed=3)
    assert [(r.model, r.tf, r.arrival) for r in r1] == [(r.model, r.tf, r.arrival) for r in r2]
    assert 60 <= len(r1) <= 140
    assert all(0 <= r.tf < 5 and r.model in models for r in r1)
    assert all(r.camera.width in (256, 512, 1024, 2048) for r in r1)
    assert np.all(np.diff([r.arrival for r in r1]) > 0)


def test_latency_stats():
    cam = S.look_at_camera((0, 0, 3), 10, 10)
    reqs = [Request(i, "m", cam, 0, arrival=0.1 * i, done=0.1 * i + 0.01 * (i + 1))
            for i in range(10)]
    st = latency_stats(reqs)
    assert abs(st["p50_ms"] - 55.0) < 1e-9 and st["requests"] == 10
    assert abs(st["mpix_per_s"] - 1000 / (0.9 + 0.1) / 1e6) < 1e-12


@pytest.mark.gpu
def test_results_same_alone_and_in_the_mix():
    import __graft_entry__
    __graft_entry__.build()
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    models = {}
    for name, n, seed in (("small", 3000, 1), ("large", 20000, 2)):
        g, _ = S.field_gaussians(n, 4, seed)
        models[name] = (dev(g.mean_v), dev(g.logscale_w), dev(g.quat))
    tfs = torch.as_tensor(S.bump_tfs(6, 5), device="cuda")
    # a burst (~40 requests within 2 ms) so that requests queue and batch
    reqs = poisson_requests(models, 6, rate=20000.0, duration=0.002, seed=9,
                            resolutions=(64, 96, 128))
    assert len(reqs) >= 20
    lim = lambda: SlotLimits(records=200_000, instances=4_000_000, pixels=1 << 20, views=6,
                             max_side=128)
    mixed = RenderServer(models, tfs, n_slots=3, max_batch=6, limits=lim(), keep_images=True)
    out_mix = mixed.run(reqs)
    assert all(r.image is not None for r in out_mix)
    assert max(mixed.batch_sizes) > 1  # requests were really batched together
    assert mixed.mixed_batches > 0     # ... across resolutions
    # each request alone: fresh copies of the requests, one at a time
    alone = [Request(r.rid, r.model, r.camera, r.tf, 0.0) for r in reqs]
    single = RenderServer(models, tfs, n_slots=1, max_batch=1, limits=lim(), keep_images=True)
    for a in alone:
        single.run([a])
    by_id = {r.rid: r for r in out_mix}
    for a in alone:
        m = by_id[a.rid]
        assert torch.equal(a.image, m.image), a.rid
    st = latency_stats(out_mix)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    # the FIFO comparison path renders the same pixels
    fifo = fifo_serve(RenderServer(models, tfs, limits=lim(), keep_images=True),
                      [Request(r.rid, r.model, r.camera, r.tf, r.arrival) for r in reqs])
    for f in fifo:
        assert torch.equal(f.image, by_id[f.rid].image)


@pytest.mark.gpu
def test_overflowing_batch_is_requeued_and_each_request_rendered_alone():
    """A batch whose tile instances overflow the slot's buffer is not waited
    for: its requests return to the queue and are rendered one at a time,
    with the same images as alone, and every request completes."""
    import __graft_entry__
    __graft_entry__.build()
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    g, _ = S.field_gaussians(20000, 4, 2)
    models = {"m": (dev(g.mean_v), dev(g.logscale_w), dev(g.quat))}
    tfs = torch.as_tensor(S.bump_tfs(4, 5), device="cuda")
    reqs = poisson_requests(models, 4, rate=20000.0, duration=0.002, seed=11,
                            resolutions=(96, 128))
    lim = lambda: SlotLimits(records=200_000, instances=120_000, pixels=1 << 20, views=6,
                             max_side=128)
    # one request alone needs 39,000-77,000 instances, any six together more
    # than 120,000
    single = RenderServer(models, tfs, n_slots=1, max_batch=1, limits=lim(), keep_images=True)
    alone = [Request(r.rid, r.model, r.camera, r.tf, 0.0) for r in reqs]
    for a in alone:
        single.run([a])
    assert all(a.status == _lib.VEG_OK for a in alone)
    per_request = max(single.inst.values())
    assert per_request * 6 > 120_000
    srv = RenderServer(models, tfs, n_slots=2, max_batch=6, limits=lim(), keep_images=True)
    for (m, w, h) in list(single.inst):  # estimates too low: batches form and overflow
        srv.inst[(m, w, h)] = 1
    out = srv.run([Request(r.rid, r.model, r.camera, r.tf, r.arrival) for r in reqs])
    assert srv.retries > 0
    by_id = {a.rid: a for a in alone}
    for r in out:
        assert r.status == _lib.VEG_OK and not np.isnan(r.done)
        assert torch.equal(r.image, by_id[r.rid].image), r.rid
