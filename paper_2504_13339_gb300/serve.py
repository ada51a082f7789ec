"""Render serving with continuous batching over resident VEG models.

Because a VEG model does not depend on the transfer function (Sec. 3.2-3.3:
colour and opacity come from the TF at render time), one resident copy of each
model serves every (view, TF) request.  The server keeps several models on
the device and admits render requests (model, camera, TF, resolution):

* a request waits in a queue until a stream slot is free; a free slot takes
  the oldest waiting request and every other waiting request for the same
  model and resolution (up to `max_batch`), and renders them as one batch:
  one projection + binning + sort over all the batch's views and one
  compositing launch in which view v uses its own TF (`veg_tf.view_tf`);
* requests that arrive while batches are on the GPU are admitted as soon as
  a slot frees, and the slots run on separate CUDA streams, so their work
  overlaps on the device (continuous batching, not a queue drained one batch
  at a time);
* device buffers are sized per (model, resolution, batch) and cached per
  slot; a byte budget bounds them (least recently used idle buffers are
  released first), which is the admission-by-memory rule;
* latency = result ready (the batch's completion event observed on the host)
  minus arrival time.

`fifo_serve` is the comparison path: one request at a time, in arrival order,
each as a plain single-view render.
"""
from __future__ import annotations

import math
import time
from collections import OrderedDict, deque
from dataclasses import dataclass, field

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

    @property
    def latency(self):
        return self.done - self.arrival


class _Buffers:
    """Device buffers for batches of up to `vmax` views of one model at one
    resolution, one image per view."""

    def __init__(self, n, vmax, width, height, capacity, device):
        self.n, self.vmax, self.W, self.H = n, vmax, width, height
        self.tiles = ((width + 15) // 16) * ((height + 15) // 16)
        nrec = n * vmax
        d = device
        self.geo = torch.empty(nrec, 4, device=d)
        self.aux = torch.empty(nrec, 4, device=d)
        self.count = torch.empty(nrec, dtype=torch.int32, device=d)
        self.rect = torch.empty(nrec, 4, dtype=torch.int16, device=d)
        self.ranges = torch.empty(vmax * self.tiles, 2, dtype=torch.int32, device=d)
        self.order = torch.empty(vmax * self.tiles, dtype=torch.int32, device=d)
        self.out = torch.empty(vmax, 1, height, width, 4, device=d)
        self.nc = torch.empty(vmax, 1, height, width, dtype=torch.int32, device=d)
        self.view_tf = torch.zeros(vmax, dtype=torch.int32, device=d)
        self.view_tf_host = torch.zeros(vmax, dtype=torch.int32).pin_memory()
        self.set_capacity(capacity, device)

    def set_capacity(self, capacity, device):
        self.capacity = int(capacity)
        ws = _lib.veg_bin_sort_workspace_size(self.n, self.vmax, self.capacity, self.W, self.H)
        self.ws = torch.empty(ws, dtype=torch.uint8, device=device)
        self.vals = torch.empty(max(1, self.capacity), dtype=torch.int32, device=device)

    def nbytes(self):
        return sum(t.numel() * t.element_size() for t in (
            self.geo, self.aux, self.count, self.rect, self.ranges, self.order, self.out, self.nc,
            self.ws, self.vals))


@dataclass
class _Slot:
    stream: torch.cuda.Stream
    event: torch.cuda.Event | None = None
    batch: list = field(default_factory=list)
    key: tuple | None = None
    bufs: "OrderedDict[tuple, _Buffers]" = field(default_factory=OrderedDict)


class RenderServer:
    """Continuous-batching render server (see module docstring)."""

    def __init__(self, models, tf_bank, n_slots=4, max_batch=8, mem_budget=64 << 30,
                 bg=(0.0, 0.0, 0.0), instances_per_view=None, keep_images=False,
                 device="cuda"):
        _lib.load()
        self.device = torch.device(device)
        self.models = {k: tuple(t.contiguous() for t in v) for k, v in models.items()}
        self.tf_bank = tf_bank.contiguous()
        self.max_batch = int(max_batch)
        self.budget = int(mem_budget)
        self.bg = tuple(float(b) for b in bg)
        self.keep = keep_images
        self.slots = [_Slot(torch.cuda.Stream(self.device)) for _ in range(n_slots)]
        # instance estimate per (model, width, height): grows on overflow
        self.inst = dict(instances_per_view or {})
        self.allocated = 0

    # -- buffers -------------------------------------------------------------
    def _capacity_for(self, model, W, H, k):
        n = self.models[model][0].shape[0]
        per_view = self.inst.get((model, W, H), 12 * n)
        return int(per_view * k * 1.25) + 4096

    def _buffers(self, slot, model, W, H):
        key = (model, W, H)
        if key in slot.bufs:
            slot.bufs.move_to_end(key)
            return slot.bufs[key]
        n = self.models[model][0].shape[0]
        cap = self._capacity_for(model, W, H, self.max_batch)
        # admission by memory: release least recently used idle buffers
        need = n * self.max_batch * 56 + cap * 16 + self.max_batch * W * H * 20
        while self.allocated + need > self.budget and self._evict_one(slot):
            pass
        b = _Buffers(n, self.max_batch, W, H, cap, self.device)
        self.allocated += b.nbytes()
        slot.bufs[key] = b
        return b

    def _evict_one(self, current):
        for s in self.slots:
            if s is not current and s.event is not None:
                continue  # busy
            for key in list(s.bufs):
                if s is current and len(s.bufs) == 1:
                    break
                b = s.bufs.pop(key)
                self.allocated -= b.nbytes()
                return True
        return False

    # -- one batch -------------------------------------------------------------
    def _launch(self, slot, batch):
        r0 = batch[0]
        W, H = r0.camera.width, r0.camera.height
        b = self._buffers(slot, r0.model, W, H)
        k = len(batch)
        g = _lib.gaussians(*self.models[r0.model])
        cams = _lib.cameras([r.camera for r in batch])
        for i, r in enumerate(batch):
            b.view_tf_host[i] = r.tf
        with torch.cuda.stream(slot.stream):
            b.view_tf[:k].copy_(b.view_tf_host[:k], non_blocking=True)
            tf = _lib.tf_desc(self.tf_bank, b.view_tf)
            s = slot.stream
            _lib.veg_project(cams, g, tf, b.geo, b.aux, b.count, b.rect, s)
            _lib.veg_bin_sort(cams, b.n, b.geo, b.count, b.rect, b.ws, b.capacity, None, b.vals,
                              b.ranges, s)
            _lib.veg_tile_order(b.ranges[:k * b.tiles], b.order, s)
            _lib.veg_composite_fwd(cams, b.n, b.geo, b.aux, b.vals, b.ranges, tf, self.bg, 1,
                                   b.out, b.nc, None, s, tile_order=b.order)
            ev = torch.cuda.Event()
            ev.record(s)
        slot.event, slot.batch, slot.key = ev, batch, (r0.model, W, H)

    def _finish(self, slot, now):
        b = slot.bufs[slot.key]
        st, m = _lib.veg_sync_status(b.ws, slot.stream)
        k = len(slot.batch)
        model, W, H = slot.key
        self.inst[(model, W, H)] = max(self.inst.get((model, W, H), 0), m // k + 1)
        if st != _lib.VEG_OK:  # capacity overflow: grow and render the batch again
            self.allocated -= b.nbytes()
            b.set_capacity(int(m * 1.25) + 4096, self.device)
            self.allocated += b.nbytes()
            batch = slot.batch
            self._launch(slot, batch)
            slot.event.synchronize()
            now = self.clock()
        for i, r in enumerate(slot.batch):
            r.done = now
            if self.keep:
                r.image = b.out[i, 0].clone()
        done = slot.batch
        slot.event, slot.batch, slot.key = None, [], None
        return done

    # -- the loop --------------------------------------------------------------
    def clock(self):
        return time.perf_counter() - self.t0

    def run(self, requests, poll_s=20e-6):
        """Serves `requests` (sorted by arrival, arrival times relative to the
        start); returns them completed.  Arrivals are released in real time."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        pending = deque()
        done = []
        nxt = 0
        self.t0 = time.perf_counter()
        while len(done) < len(reqs):
            now = self.clock()
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                pending.append(reqs[nxt])
                nxt += 1
            for s in self.slots:
                if s.event is not None and s.event.query():
                    done.extend(self._finish(s, self.clock()))
            for s in self.slots:
                if s.event is None and pending:
                    head = pending[0]
                    key = (head.model, head.camera.width, head.camera.height)
                    batch = [r for r in pending
                             if (r.model, r.camera.width, r.camera.height) == key][:self.max_batch]
                    for r in batch:
                        pending.remove(r)
                    self._launch(s, batch)
            if not pending and nxt < len(reqs):
                wait = reqs[nxt].arrival - self.clock()
                if wait > 1e-3:
                    time.sleep(min(wait, 1e-3) * 0.5)
            elif poll_s:
                time.sleep(poll_s)
        return reqs


def fifo_serve(server: RenderServer, requests, poll_s=20e-6):
    """One request at a time in arrival order on one stream (the plain path)."""
    saved = (server.max_batch, server.slots)
    server.slots = server.slots[:1]
    server.max_batch = 1
    try:
        return server.run(requests, poll_s)
    finally:
        server.max_batch, server.slots = saved


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
