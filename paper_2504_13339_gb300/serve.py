"""Render serving with continuous batching over resident VEG models.

Because a VEG model does not depend on the transfer function (Sec. 3.2-3.3:
colour and opacity come from the TF at render time), one resident copy of each
model serves every (view, TF) request.  The server keeps several models on
the device and admits render requests (model, camera, TF, resolution):

* Memory: each stream slot owns one fixed set of device buffers, allocated
  up front (records, tile instances, pixels, views).  The number of slots is
  what the memory budget admits; nothing is allocated while serving.
* Batching: a free slot takes the oldest waiting request and every other
  waiting request for the same model, at any resolution, that still fits
  its buffers (records = views x Gaussians, pixels, estimated tile
  instances), and renders them as one batch: one projection + binning + sort
  over all the batch's views, whose image sizes may differ, and one
  compositing launch in which view v uses its own TF (`veg_tf.view_tf`) and
  writes its own image.
* Continuity: requests that arrive while batches run are admitted as soon as
  a slot frees; slots run on separate CUDA streams, so their work overlaps
  on the device.
* Latency = result ready (the batch's completion event observed on the host)
  minus arrival time.  The tile instances of each (model, resolution) are
  learned from completed batches (a batch's count is shared over its
  requests in proportion to their pixels; a batch's estimate sums its
  requests');
  a batch that overflowed its instance buffer is not waited for again: its
  requests go back to the front of the queue, each to be rendered alone
  when a slot frees, and a request whose own render still overflows carries
  that status.
* Memory admission is by slots: the server builds as many slots as the
  memory budget holds (at least one), and a request is admitted into a
  batch when the batch's records, pixels and estimated instances fit the
  slot's fixed buffers; nothing is allocated while serving.
* Batching window (optional, `batch_window_ms` > 0): a free slot launches a
  model's waiting requests only once they are `min_batch` or more, fill a
  batch, or the oldest of them has waited the window; until then the slot
  stays free for another model.  This trades up to a window of latency for
  larger batches when arrivals are sparse (the immediate policy launches
  whatever waits as soon as a slot frees, which at moderate rates is one
  request).
* Batches across models (optional, `cross_model`): a batch may hold views
  of different models (`veg_project_views`: each view projects its own
  model into records of a common stride, the largest model's size; a
  smaller model's remaining records touch no tile), so waiting requests
  batch whatever model they ask for, as long as at most half of a batch's
  records are such padding.  With the window, all waiting requests form
  one group.

`fifo_serve` is the comparison path: one request at a time, in arrival order,
each as a plain single-view render.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field, replace

import numpy as np
import torch

from . import _lib


@dataclass
class Request:
    rid: int
    model: str
    camera: object  # scenes.Camera
    tf: int          # index into the server's TF bank
    arrival: float   # seconds, on the server clock
    done: float = math.nan
    image: torch.Tensor | None = None  # [H][W][4] when kept
    status: int = 0  # VEG_OK, or VEG_ERR_CAPACITY if even its own render overflowed
    solo: bool = False  # its batch overflowed: render it alone

    @property
    def latency(self):
        return self.done - self.arrival


@dataclass
class SlotLimits:
    records: int = 12_000_000    # views x Gaussians per batch
    instances: int = 160_000_000
    pixels: int = 16 << 20       # views x width x height per batch
    views: int = 8
    max_side: int = 2048


class _SlotBuffers:
    """One slot's device memory, reused by every batch it renders."""

    def __init__(self, lim: SlotLimits, device):
        d = device
        self.lim = lim
        R, P, V = lim.records, lim.pixels, lim.views
        tiles = V * ((lim.max_side + 15) // 16) ** 2
        self.geo = torch.empty(R, 4, device=d)
        self.aux = torch.empty(R, 4, device=d)
        self.count = torch.empty(R, dtype=torch.int32, device=d)
        self.rect = torch.empty(R, 4, dtype=torch.int16, device=d)
        self.ranges = torch.empty(tiles, 2, dtype=torch.int32, device=d)
        self.order = torch.empty(tiles, dtype=torch.int32, device=d)
        self.out = torch.empty(P * 4, device=d)
        self.nc = torch.empty(P, dtype=torch.int32, device=d)
        self.view_tf = torch.zeros(V, dtype=torch.int32, device=d)
        self.view_tf_host = torch.zeros(V, dtype=torch.int32).pin_memory()
        self.n_inst = torch.zeros(1, dtype=torch.int64, device=d)
        # the workspace layout depends only on records and capacity
        ws = _lib.veg_bin_sort_workspace_size(R, 1, lim.instances, lim.max_side, lim.max_side)
        self.ws = torch.empty(ws, dtype=torch.uint8, device=d)
        self.vals = torch.empty(lim.instances, dtype=torch.int32, device=d)

    def nbytes(self):
        return sum(t.numel() * t.element_size() for t in (
            self.geo, self.aux, self.count, self.rect, self.ranges, self.order, self.out, self.nc,
            self.ws, self.vals))


@dataclass
class _Slot:
    stream: torch.cuda.Stream
    bufs: _SlotBuffers
    event: torch.cuda.Event | None = None
    batch: list = field(default_factory=list)
    offsets: list = field(default_factory=list)  # first pixel of each request's image


class RenderServer:
    """Continuous-batching render server (see module docstring)."""

    def __init__(self, models, tf_bank, n_slots=4, max_batch=8, limits=None,
                 mem_budget=None, bg=(0.0, 0.0, 0.0), keep_images=False, device="cuda",
                 batch_window_ms=0.0, min_batch=2, cross_model=False):
        _lib.load()
        self.device = torch.device(device)
        self.models = {k: tuple(t.contiguous() for t in v) for k, v in models.items()}
        self.tf_bank = tf_bank.contiguous()
        self.lim = replace(limits or SlotLimits())  # the caller's limits stay as given
        self.lim.views = min(self.lim.views, int(max_batch))
        self.bg = tuple(float(b) for b in bg)
        self.keep = keep_images
        self.slots = []
        used = 0
        for _ in range(n_slots):
            b = _SlotBuffers(self.lim, self.device)
            if mem_budget is not None and self.slots and used + b.nbytes() > mem_budget:
                break  # admission by memory: no more slots than fit (at least one)
            used += b.nbytes()
            self.slots.append(_Slot(torch.cuda.Stream(self.device), b))
        self.bytes = used
        self.inst = {}  # (model, W, H) -> tile instances of one view (largest seen)
        self.batch_sizes = []
        self.mixed_batches = 0  # batches holding more than one resolution
        self.retries = 0  # requests put back after their batch overflowed
        self.multi_model_batches = 0  # batches holding more than one model
        self.window = max(0.0, float(batch_window_ms)) * 1e-3
        self.min_batch = max(1, int(min_batch))
        self.cross_model = bool(cross_model)

    def _est(self, model, W, H):
        n = self.models[model][0].shape[0]
        return self.inst.get((model, W, H), min(16 * n, self.lim.instances))

    def _fits(self, batch):
        """The batch's views, records (views x the largest model's size),
        pixels and estimated instances fit a slot's buffers; across models,
        at most half the records are padding (a small model's view beside a
        large one projects the large one's record count)."""
        sizes = [self.models[r.model][0].shape[0] for r in batch]
        n = max(sizes)
        k = len(batch)
        if k > 1 and k * n > 2 * sum(sizes):
            return False
        pix = sum(r.camera.width * r.camera.height for r in batch)
        inst = sum(self._est(r.model, r.camera.width, r.camera.height) for r in batch)
        return (k <= self.lim.views and k * n <= self.lim.records and pix <= self.lim.pixels
                and inst <= self.lim.instances)

    # -- one batch -------------------------------------------------------------
    def _launch(self, slot, batch):
        r0 = batch[0]
        b = slot.bufs
        k = len(batch)
        one_model = all(r.model == r0.model for r in batch)
        n = max(self.models[r.model][0].shape[0] for r in batch)
        g = _lib.gaussians(*self.models[r0.model])
        cams = _lib.cameras([r.camera for r in batch])
        offsets, tiles = [0], 0
        for i, r in enumerate(batch):
            W, H = r.camera.width, r.camera.height
            offsets.append(offsets[-1] + W * H)
            tiles += ((W + 15) // 16) * ((H + 15) // 16)
            b.view_tf_host[i] = r.tf
        npix = offsets[-1]
        s = slot.stream
        with torch.cuda.stream(s):
            b.view_tf[:k].copy_(b.view_tf_host[:k], non_blocking=True)
            tf = _lib.tf_desc(self.tf_bank, b.view_tf)
            out = b.out[:npix * 4]
            nc = b.nc[:npix]
            if one_model:
                _lib.veg_project(cams, g, tf, b.geo, b.aux, b.count, b.rect, s)
            else:
                _lib.veg_project_views(cams, [_lib.gaussians(*self.models[r.model])
                                              for r in batch], n, tf, b.geo, b.aux, b.count,
                                       b.rect, s)
            _lib.veg_bin_sort(cams, n, b.geo, b.count, b.rect, b.ws, self.lim.instances, None,
                              b.vals, b.ranges, s)
            _lib.veg_tile_order(b.ranges[:tiles], b.order, s)
            _lib.veg_composite_fwd(cams, n, b.geo, b.aux, b.vals, b.ranges, tf, self.bg, 1, out,
                                   nc, None, s, tile_order=b.order)
            ev = torch.cuda.Event()
            ev.record(s)
        slot.event, slot.batch, slot.offsets = ev, batch, offsets
        self.batch_sizes.append(k)
        self.mixed_batches += len({(r.camera.width, r.camera.height) for r in batch}) > 1
        self.multi_model_batches += not one_model

    def _finish(self, slot):
        """Completes a slot's finished batch; returns (completed requests,
        requests to render again alone)."""
        b = slot.bufs
        st, m = _lib.veg_sync_status(b.ws, slot.stream)  # the stream is already done
        batch, offsets = slot.batch, slot.offsets
        slot.event, slot.batch, slot.offsets = None, [], []
        # the instances per view, shared over the batch in proportion to pixels
        for i, r in enumerate(batch):
            key = (r.model, r.camera.width, r.camera.height)
            share = m * (offsets[i + 1] - offsets[i]) / offsets[-1]
            self.inst[key] = max(self.inst.get(key, 0), int(share * 1.2) + 1)
        if st != _lib.VEG_OK and len(batch) > 1:
            for r in batch:
                r.solo = True
            self.retries += len(batch)
            return [], batch
        now = self.clock()
        for i, r in enumerate(batch):
            r.done = now
            r.status = st
            if self.keep:
                W, H = r.camera.width, r.camera.height
                r.image = b.out[offsets[i] * 4:offsets[i + 1] * 4].view(H, W, 4).clone()
        return batch, []

    # -- the loop --------------------------------------------------------------
    def clock(self):
        return time.perf_counter() - self.t0

    def _gather(self, pending, head):
        """`head` and every later waiting request of its model (of any model
        with cross_model) that fits."""
        batch = [head]
        if not head.solo:
            for r in pending:
                if r is not head and not r.solo and (self.cross_model or r.model == head.model) \
                        and self._fits(batch + [r]):
                    batch.append(r)
        return batch

    def _take_batch(self, pending):
        """The next batch to launch, removed from `pending`, or None when the
        batching window holds every model's requests back."""
        if self.window <= 0.0:
            batch = self._gather(pending, pending[0])
        else:
            now, batch, seen = self.clock(), None, set()
            for r in pending:  # oldest first: the first model ready goes
                if (r.model in seen or (self.cross_model and seen)) and not r.solo:
                    continue
                seen.add(r.model)
                b = self._gather(pending, r)
                # no room for one more request like the last: launch now
                full = len(b) >= self.lim.views or not self._fits(b + [b[-1]])
                if r.solo or full or len(b) >= self.min_batch or now - r.arrival >= self.window:
                    batch = b
                    break
            if batch is None:
                return None
        for r in batch:
            pending.remove(r)
        return batch

    def run(self, requests, poll_s=20e-6):
        """Serves `requests` (arrival times relative to the start, released in
        real time); returns them completed."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        pending = deque()
        n_done = 0
        nxt = 0
        self.t0 = time.perf_counter()
        while n_done < len(reqs):
            now = self.clock()
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                pending.append(reqs[nxt])
                nxt += 1
            for s in self.slots:
                if s.event is not None and s.event.query():
                    done, retry = self._finish(s)
                    n_done += len(done)
                    pending.extendleft(reversed(retry))
            for s in self.slots:
                if s.event is None and pending:
                    batch = self._take_batch(pending)
                    if batch is None:
                        break  # the window holds the waiting requests back
                    self._launch(s, batch)
            if not pending and nxt < len(reqs) and all(s.event is None for s in self.slots):
                wait = reqs[nxt].arrival - self.clock()
                if wait > 2e-4:
                    time.sleep(wait * 0.5)
            elif poll_s:
                time.sleep(poll_s)
        return reqs


def fifo_serve(server: RenderServer, requests, poll_s=20e-6):
    """One request at a time in arrival order on one stream (the plain path)."""
    saved = (server.lim.views, server.slots)
    server.slots = server.slots[:1]
    server.lim.views = 1
    try:
        return server.run(requests, poll_s)
    finally:
        server.lim.views, server.slots = saved


def latency_stats(reqs):
    lat = np.array([r.latency for r in reqs]) * 1e3
    pix = sum(r.camera.width * r.camera.height for r in reqs)
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "mpix_per_s": pix / span / 1e6, "requests": len(reqs)}


def poisson_requests(models, n_tf, rate, duration, seed, resolutions=(256, 512, 1024, 2048),
                     radius=3.0, el_max=30.0):
    """Seeded Poisson arrivals: uniformly random model, orbit view, TF index
    and square resolution."""
    from . import scenes as S
    rng = np.random.default_rng(seed)
    t, out, rid = 0.0, [], 0
    names = list(models)
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        res = int(rng.choice(resolutions))
        cam = S.orbit_camera(rng.uniform(0, 360), rng.uniform(-el_max, el_max), radius, res, res)
        out.append(Request(rid, names[rng.integers(len(names))], cam, int(rng.integers(n_tf)), t))
        rid += 1
    return out
