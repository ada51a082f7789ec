"""Render serving with continuous batching over resident VEG models.

Because a VEG model does not depend on the transfer function (Sec. 3.2-3.3:
colour and opacity come from the TF at render time), one resident copy of each
model serves every (view, TF) request.  The server keeps several models on
the device and admits render requests (model, camera, TF, resolution):

* Memory: each stream slot owns one fixed set of device buffers, allocated
  up front (records, tile instances, pixels, views).  The number of slots is
  what the memory budget admits; nothing is allocated while serving.
* Batching: a free slot takes the oldest waiting request and every other
  waiting request for the same model and resolution that still fits its
  buffers (records = views x Gaussians, pixels, estimated tile instances),
  and renders them as one batch: one projection + binning + sort over all
  the batch's views and one compositing launch in which view v uses its own
  TF (`veg_tf.view_tf`).
* Continuity: requests that arrive while batches run are admitted as soon as
  a slot frees; slots run on separate CUDA streams, so their work overlaps
  on the device.
* Latency = result ready (the batch's completion event observed on the host)
  minus arrival time.  The per-(model, resolution) instance estimate is
  learned from completed batches; a batch that overflowed its instance
  buffer is rendered again one request at a time, and a request whose own
  render still overflows carries that status.

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


class RenderServer:
    """Continuous-batching render server (see module docstring)."""

    def __init__(self, models, tf_bank, n_slots=4, max_batch=8, limits=None,
                 mem_budget=None, bg=(0.0, 0.0, 0.0), keep_images=False, device="cuda"):
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
        self.inst = {}  # (model, W, H) -> tile instances per view (largest seen)
        self.batch_sizes = []

    def _est(self, model, W, H):
        n = self.models[model][0].shape[0]
        return self.inst.get((model, W, H), min(16 * n, self.lim.instances))

    def _fits(self, model, W, H, k):
        n = self.models[model][0].shape[0]
        return (k <= self.lim.views and k * n <= self.lim.records
                and k * W * H <= self.lim.pixels
                and k * self._est(model, W, H) <= self.lim.instances)

    # -- one batch -------------------------------------------------------------
    def _launch(self, slot, batch):
        r0 = batch[0]
        W, H = r0.camera.width, r0.camera.height
        b = slot.bufs
        k = len(batch)
        n = self.models[r0.model][0].shape[0]
        g = _lib.gaussians(*self.models[r0.model])
        cams = _lib.cameras([r.camera for r in batch])
        tiles = ((W + 15) // 16) * ((H + 15) // 16)
        for i, r in enumerate(batch):
            b.view_tf_host[i] = r.tf
        s = slot.stream
        with torch.cuda.stream(s):
            b.view_tf[:k].copy_(b.view_tf_host[:k], non_blocking=True)
            tf = _lib.tf_desc(self.tf_bank, b.view_tf)
            out = b.out[:k * H * W * 4].view(k, 1, H, W, 4)
            nc = b.nc[:k * H * W].view(k, 1, H, W)
            _lib.veg_project(cams, g, tf, b.geo, b.aux, b.count, b.rect, s)
            _lib.veg_bin_sort(cams, n, b.geo, b.count, b.rect, b.ws, self.lim.instances, None,
                              b.vals, b.ranges, s)
            _lib.veg_tile_order(b.ranges[:k * tiles], b.order, s)
            _lib.veg_composite_fwd(cams, n, b.geo, b.aux, b.vals, b.ranges, tf, self.bg, 1, out,
                                   nc, None, s, tile_order=b.order)
            ev = torch.cuda.Event()
            ev.record(s)
        slot.event, slot.batch = ev, batch
        self.batch_sizes.append(k)
        return out

    def _finish(self, slot):
        b = slot.bufs
        st, m = _lib.veg_sync_status(b.ws, slot.stream)  # the stream is already done
        batch = slot.batch
        r0 = batch[0]
        key = (r0.model, r0.camera.width, r0.camera.height)
        self.inst[key] = max(self.inst.get(key, 0), int(m / len(batch) * 1.2) + 1)
        if st != _lib.VEG_OK:  # overflow: render the batch again one request at a time
            for r in batch:
                out = self._launch(slot, [r])
                slot.event.synchronize()
                r.status = _lib.veg_sync_status(b.ws, slot.stream)[0]
                self._complete(slot, [r], out)
        else:
            H, W = r0.camera.height, r0.camera.width
            self._complete(slot, batch, b.out[:len(batch) * H * W * 4].view(len(batch), 1, H, W,
                                                                            4))
        slot.event, slot.batch = None, []
        return batch

    def _complete(self, slot, batch, out):
        now = self.clock()
        for i, r in enumerate(batch):
            r.done = now
            if self.keep:
                r.image = out[i, 0].clone()

    # -- the loop --------------------------------------------------------------
    def clock(self):
        return time.perf_counter() - self.t0

    def _take_batch(self, pending):
        head = pending[0]
        key = (head.model, head.camera.width, head.camera.height)
        batch = [head]
        for r in list(pending)[1:]:
            if (r.model, r.camera.width, r.camera.height) == key and \
                    self._fits(head.model, key[1], key[2], len(batch) + 1):
                batch.append(r)
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
                    n_done += len(self._finish(s))
            for s in self.slots:
                if s.event is None and pending:
                    self._launch(s, self._take_batch(pending))
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
