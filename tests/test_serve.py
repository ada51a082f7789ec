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


def _policy_server(window_ms, min_batch=2, views=8):
    """A RenderServer with only what the batching policy reads (no device)."""
    import time
    srv = object.__new__(RenderServer)
    srv.models = {"a": (torch.empty(100, 4),), "b": (torch.empty(100, 4),)}
    srv.lim = SlotLimits(records=100 * views, instances=10**9, pixels=1 << 30, views=views,
                         max_side=64)
    srv.inst = {}
    srv.window = window_ms * 1e-3
    srv.min_batch = min_batch
    srv.cross_model = False
    srv.t0 = time.perf_counter()
    return srv


def test_batching_window_policy():
    """With a window, a model's requests wait for a partner until the oldest
    has waited the window; a pair, a full batch or a retry goes at once;
    another model that is ready goes first; without a window the head's
    batch goes immediately."""
    from collections import deque
    cam = S.look_at_camera((0, 0, 3), 32, 32)
    R = lambda i, m, t, solo=False: Request(i, m, cam, 0, arrival=t, solo=solo)
    srv = _policy_server(10.0)
    srv.clock = lambda: 0.004
    q = deque([R(0, "a", 0.0)])
    assert srv._take_batch(q) is None and len(q) == 1  # 4 ms old: held
    srv.clock = lambda: 0.0101
    assert [r.rid for r in srv._take_batch(q)] == [0] and not q  # the window ran out
    srv.clock = lambda: 0.002
    q = deque([R(1, "a", 0.0), R(2, "b", 0.0005), R(3, "b", 0.001), R(4, "a", 0.0015)])
    assert [r.rid for r in srv._take_batch(q)] == [1, 4]  # a has two: both go
    q = deque([R(5, "a", 0.0), R(6, "b", 0.0005), R(7, "b", 0.001)])
    assert [r.rid for r in srv._take_batch(q)] == [6, 7]  # a alone waits, b's pair goes
    assert [r.rid for r in q] == [5]
    q = deque([R(8, "a", 0.0015, solo=True)])
    assert [r.rid for r in srv._take_batch(q)] == [8]  # a retry goes alone at once
    full = _policy_server(10.0, min_batch=99, views=3)
    full.clock = lambda: 0.001
    q = deque([R(10 + i, "a", 0.0) for i in range(4)])
    assert [r.rid for r in full._take_batch(q)] == [10, 11, 12]  # a full batch goes
    now = _policy_server(0.0)
    now.clock = lambda: 0.0
    q = deque([R(20, "a", 0.0), R(21, "b", 0.0), R(22, "a", 0.0)])
    assert [r.rid for r in now._take_batch(q)] == [20, 22]
    # across models: every waiting request is one group
    cross = _policy_server(10.0)
    cross.cross_model = True
    cross.clock = lambda: 0.002
    q = deque([R(30, "a", 0.0), R(31, "b", 0.001)])
    assert [r.rid for r in cross._take_batch(q)] == [30, 31] and not q
    q = deque([R(32, "b", 0.0)])
    assert cross._take_batch(q) is None


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
    # the windowed policy, on sparse arrivals: requests wait for partners,
    # batches form, every image is the same as alone
    sparse = poisson_requests(models, 6, rate=400.0, duration=0.1, seed=10,
                              resolutions=(64, 96, 128))
    win = RenderServer(models, tfs, n_slots=3, max_batch=6, limits=lim(), keep_images=True,
                       batch_window_ms=30.0)
    out_win = win.run([Request(r.rid, r.model, r.camera, r.tf, r.arrival) for r in sparse])
    assert np.mean(win.batch_sizes) >= 1.5
    single2 = RenderServer(models, tfs, n_slots=1, max_batch=1, limits=lim(), keep_images=True)
    for r in out_win:
        a = Request(r.rid, r.model, r.camera, r.tf, 0.0)
        single2.run([a])
        assert torch.equal(a.image, r.image), r.rid
    # across models: batches mix the two models, each image as alone
    cross = RenderServer(models, tfs, n_slots=3, max_batch=6, limits=lim(), keep_images=True,
                         batch_window_ms=30.0, cross_model=True)
    out_x = cross.run([Request(r.rid, r.model, r.camera, r.tf, r.arrival) for r in sparse])
    assert cross.multi_model_batches > 0 and np.mean(cross.batch_sizes) >= 2.0
    for r in out_x:
        a = Request(r.rid, r.model, r.camera, r.tf, 0.0)
        single2.run([a])
        assert torch.equal(a.image, r.image), r.rid


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
