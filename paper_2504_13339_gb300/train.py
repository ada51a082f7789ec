"""Opacity-guided training of VEG models (Sec. 4.2) on the GPU.

Every iteration picks a random (camera, opacity map) pair of the training
set, renders the model for it (projection, Blinn-Phong shading with the
camera's headlight, binning, compositing), evaluates (1 - lambda) L1 +
lambda (1 - SSIM) against the matching target image, runs the backward pass
through compositing, shading and projection, and takes one Adam step on the
raw parameters, which also writes the activated values for the next render.
All of it runs in libveg.so; PyTorch holds the buffers.

The opacity maps divide the scalar range into K steps, one map centred in
each step with linear fall-off of slope K (reading R13: the colour is shared,
the maps tabulated like every transfer function).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import _lib
from .render import SplatPipeline, headlight_dirs

LAMBDA_SSIM = 0.2


def opacity_guided_luts(K, rgb, slope=None) -> np.ndarray:
    """K RGBA tables [K][L][4]: colour `rgb` (L, 3); map k's opacity
    max(0, 1 - slope |x - (k + 1/2)/K|) at x_j = j/(L-1), slope K by default."""
    rgb = np.asarray(rgb, np.float32)
    L = rgb.shape[0]
    s = float(K) if slope is None else float(slope)
    x = np.arange(L, dtype=np.float64) / (L - 1)
    luts = np.empty((K, L, 4), np.float32)
    for k in range(K):
        centre = (k + 0.5) / K
        luts[k, :, :3] = rgb
        luts[k, :, 3] = np.clip(1.0 - s * np.abs(x - centre), 0.0, None)
    return luts


def default_lr(extent=1.0, lighting=True) -> np.ndarray:
    """Learning rates [5][4] per packed array and component: the paper's
    0.00025 (scalar) and 0.025 (weight) and, following the 3D Gaussian
    splatting defaults it adopts, 1.6e-4 x scene extent (mean), 0.005
    (log-scale), 0.001 (rotation); 0.001 for normals, shininess and the
    lighting coefficients (our choice: the paper does not give them)."""
    lr = np.zeros((5, 4))
    lr[0] = [1.6e-4 * extent] * 3 + [2.5e-4]
    lr[1] = [5e-3] * 3 + [2.5e-2]
    lr[2] = [1e-3] * 4
    if lighting:
        lr[3] = [1e-3] * 4
        lr[4] = [1e-3] * 3 + [0.0]
    return lr


def _logit(p):
    p = np.clip(np.asarray(p, np.float64), 1e-4, 1.0 - 1e-4)
    return np.log(p) - np.log1p(-p)


class TrainParams:
    """Raw parameters, gradients, Adam moments and the rendered arrays of a
    model with n Gaussians, all device-resident."""

    def __init__(self, g, lighting=None, device="cuda"):
        dev = torch.device(device)
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=dev)
        mv = np.array(g.mean_v, np.float64)
        lw = np.array(g.logscale_w, np.float64)
        mv[:, 3] = _logit(mv[:, 3])
        lw[:, 3] = _logit(lw[:, 3])
        self.n = g.n
        self.lit = lighting is not None
        self.raw = [t(mv), t(lw), t(g.quat),
                    t(lighting.normal_beta) if self.lit else None,
                    t(lighting.k_ads) if self.lit else None]
        # rendered arrays: (mu, sigmoid(v_raw)), (log-scale, sigmoid(w_raw)); the
        # quaternion and the lighting arrays are rendered as stored
        self.mean_v = t(g.mean_v)
        self.logscale_w = t(g.logscale_w)
        self.grads = [None if r is None else torch.zeros_like(r) for r in self.raw]
        self.m = [None if r is None else torch.zeros_like(r) for r in self.raw]
        self.v = [None if r is None else torch.zeros_like(r) for r in self.raw]
        self.step = 0
        self.counter = None  # device step counter (use_device_counter)
        self.flat_grads = None  # one buffer behind the gradients (use_flat_gradients)
        # the full-capacity arrays behind the row views above:
        # (rows, raw, m, v, mean_v, logscale_w) and the gradients' (rows, grads)
        self.store = (self.n, self.raw, self.m, self.v, self.mean_v, self.logscale_w)
        self._grad_store = (self.n, self.grads)
        self._arrays = _lib.adam_arrays(self.raw, self.grads, self.m, self.v,
                                        (self.mean_v, self.logscale_w))

    def rendered(self):
        return self.mean_v, self.logscale_w, self.raw[2]

    def zero_grad(self):
        for gb in self.grads:
            if gb is not None:
                gb.zero_()

    def adam(self, lr, stream=None):
        self.step += 1
        if self.counter is not None:
            _lib.veg_adam_step_counted(self._arrays, self.n, lr, self.counter, stream=stream)
        else:
            _lib.veg_adam_step(self._arrays, self.n, lr, self.step, stream=stream)

    def use_flat_gradients(self):
        """Re-points the gradient arrays into one flat buffer `flat_grads`
        (zeroed), so that a data-parallel step all-reduces them with one
        collective."""
        if self.flat_grads is None:
            live = [g for g in self.grads if g is not None]
            flat = torch.zeros(sum(g.numel() for g in live), device=live[0].device)
            off, grads = 0, []
            for g in self.grads:
                if g is None:
                    grads.append(None)
                    continue
                grads.append(flat[off:off + g.numel()].view_as(g))
                off += g.numel()
            self.flat_grads, self.grads = flat, grads
            self._grad_store = (self.n, grads)
            self._arrays = _lib.adam_arrays(self.raw, self.grads, self.m, self.v,
                                            (self.mean_v, self.logscale_w))
        return self.flat_grads

    def use_device_counter(self):
        """Keeps the Adam step number on the device (veg_adam_step_counted), so
        that a captured CUDA graph can replay the step; the host count `step`
        then only advances with eager calls."""
        if self.counter is None:
            dev = self.raw[0].device
            self.counter = torch.zeros(2, dtype=torch.int64, device=dev)
            self.counter[0] = self.step
        return self.counter

    def replace(self, n, store):
        """Adopts the first n rows of `store` = (rows, raw, m, v, mean_v,
        logscale_w), full-capacity arrays (after densification); gradients
        restart at zero, in their own storage while it has room.  Returns the
        storage given up."""
        n = int(n)
        rows, raw, m, v, mean_v, logscale_w = store
        if n > rows:
            raise ValueError("replace: n exceeds the storage's rows")
        cut = lambda t: None if t is None else t[:n]
        old, self.store, self.n = self.store, store, n
        self.raw, self.m, self.v = [cut(t) for t in raw], [cut(t) for t in m], [cut(t) for t in v]
        self.mean_v, self.logscale_w = mean_v[:n], logscale_w[:n]
        grows, gfull = self._grad_store
        if self.flat_grads is not None:
            # one contiguous [n][4] run per array, so the flat buffer stays whole
            live = sum(r is not None for r in raw)
            if self.flat_grads.numel() < live * n * 4:
                self.flat_grads = torch.zeros(live * (n + n // 4) * 4,
                                              device=self.flat_grads.device)
            off, gfull = 0, []
            for r in raw:
                if r is None:
                    gfull.append(None)
                    continue
                gfull.append(self.flat_grads[off:off + n * 4].view(n, 4))
                off += n * 4
            self.flat_grads = self.flat_grads[:off] if off else self.flat_grads
            grows = n
            self._grad_store = (grows, gfull)
        elif n > grows:
            grows = n + n // 4
            gfull = [None if r is None else torch.empty(grows, 4, device=r.device)
                     for r in raw]
            self._grad_store = (grows, gfull)
        self.grads = [cut(t) for t in gfull]
        self.zero_grad()
        self._arrays = _lib.adam_arrays(self.raw, self.grads, self.m, self.v,
                                        (self.mean_v, self.logscale_w))
        return old


def scene_extent(cams) -> float:
    """1.1 x the largest distance of a camera centre from the centres'
    centroid (the extent used by the densification size rule)."""
    c = np.stack([-np.asarray(k.world_to_cam, np.float64)[:, :3].T
                  @ np.asarray(k.world_to_cam, np.float64)[:, 3] for k in cams])
    return 1.1 * float(np.linalg.norm(c - c.mean(0), axis=1).max())


class DensityControl:
    """Adaptive density control (Sec. 4.2, after 3D Gaussian splatting):
    the positional-gradient statistic is accumulated after every backward
    pass from `start` to `stop`; every `every` iterations in that window
    Gaussians are cloned, split or pruned (veg_densify)."""

    def __init__(self, extent, start=500, stop=20000, every=100, grad_threshold=2e-4,
                 dense_fraction=0.01, prune_weight=0.005, split_factor=1.6, seed=0,
                 device="cuda"):
        self.start, self.stop, self.every = int(start), int(stop), int(every)
        self.cfg = _lib.veg_density_config(
            grad_threshold, math.log(dense_fraction * extent),
            math.log(prune_weight) - math.log1p(-prune_weight), math.log(split_factor))
        self.device = torch.device(device)
        self.gen = torch.Generator(device=self.device)
        self.gen.manual_seed(seed)
        self.accum = self.count = None
        self.n_out = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.history = []
        # buffers kept between densifications: the statistic's storage, the
        # spare parameter storage that receives the next output (the storage
        # the parameters give up becomes the next spare), draws, workspace
        self._stat = None
        self._spare = None
        self._z = None
        self._ws = None

    def reset(self, n):
        if self._stat is None or self._stat[0].numel() < n:
            rows = n + n // 4
            self._stat = (torch.empty(rows, device=self.device),
                          torch.empty(rows, dtype=torch.int32, device=self.device))
        self.accum, self.count = self._stat[0][:n], self._stat[1][:n]
        self.accum.zero_()
        self.count.zero_()

    def _output_store(self, P, rows):
        """Parameter storage with at least `rows` rows for veg_densify's output."""
        s = self._spare
        if s is None or s[0] < rows or [t is None for t in s[1]] != [t is None for t in P.raw]:
            cap = rows + rows // 4
            new = lambda r: None if r is None else torch.empty(cap, 4, device=self.device)
            s = (cap, [new(r) for r in P.raw], [new(r) for r in P.raw], [new(r) for r in P.raw],
                 torch.empty(cap, 4, device=self.device), torch.empty(cap, 4, device=self.device))
        self._spare = None
        return s

    def active(self, it):
        return self.start <= it <= self.stop

    def due(self, it):
        return self.active(it) and it > self.start and it % self.every == 0

    def accumulate(self, pipe, P, stream=None):
        if self.accum is None or self.accum.numel() != P.n:
            self.reset(P.n)
        _lib.veg_grad_stats_accumulate(pipe.grad2d, pipe.tiles, P.n, pipe.V, pipe.W, pipe.H,
                                       self.accum, self.count, stream)

    def apply(self, P, stream=None):
        """Clone / split / prune; replaces P's arrays (one host sync to read
        the new count).  Returns the new number of Gaussians."""
        n = P.n
        if self.accum is None or self.accum.numel() != n:
            self.reset(n)
        store = self._output_store(P, 2 * n)
        cap, raw, m, v, mean_v, logscale_w = store
        if self._z is None or self._z.numel() < 6 * n:
            self._z = torch.empty(6 * (n + n // 4), device=self.device)
        z = self._z[:6 * n].view(n, 2, 3)
        torch.randn(n, 2, 3, generator=self.gen, out=z)
        wsb = max(_lib.veg_densify_workspace_size(n), 1)
        if self._ws is None or self._ws.numel() < wsb:
            self._ws = torch.empty(wsb + wsb // 4, dtype=torch.uint8, device=self.device)
        src = _lib.adam_arrays(P.raw, P.grads, P.m, P.v)
        dst = _lib.adam_arrays(raw, [None] * 5, m, v, (mean_v, logscale_w))
        _lib.veg_densify(src, n, self.accum, self.count, z, self.cfg, dst, cap, self.n_out,
                         None, self._ws, stream)
        n_new = int(self.n_out.item())
        self._spare = P.replace(n_new, store)
        self.reset(n_new)
        self.history.append((n, n_new))
        return n_new


class OpacityGuidedTrainer:
    """Random (view, opacity map) per iteration, L1 + SSIM loss, Adam.

    cams: the training views (same size); luts: device tensor [K][L][4];
    targets: device tensor [V][K][H][W][4] of ground-truth images.  With
    lighting (params.lit) every view is shaded with its headlight."""

    def __init__(self, params: TrainParams, cams, luts, targets, lr=None, lam=LAMBDA_SSIM,
                 seed=0, capacity=None, bg=(0.0, 0.0, 0.0), density: DensityControl = None,
                 native=True):
        self.P = params
        self.density = density
        self.it = 0
        self.capacity = capacity
        self.native = bool(native)
        self._args = None
        self._c_all = None
        self.cams = list(cams)
        self.luts = luts
        self.targets = targets
        self.K = luts.shape[0]
        self.lam = float(lam)
        self.lr = default_lr(lighting=params.lit) if lr is None else np.asarray(lr)
        self.rng = np.random.default_rng(seed)
        self.bg = bg
        self.lights = headlight_dirs(self.cams).astype(np.float32)
        self.pipe = SplatPipeline(params.n, self.cams[:1], n_tf=1, capacity=capacity)
        self.c_cams = [_lib.cameras([c]) for c in self.cams]
        H, W = self.cams[0].height, self.cams[0].width
        dev = self.pipe.device
        self.loss = torch.zeros(3, device=dev)
        self.loss_ws = torch.empty(_lib.veg_l1_ssim_loss_workspace_size(1, H, W),
                                   dtype=torch.uint8, device=dev)

    def render(self, view, k, stream=None):
        p, P = self.pipe, self.P
        p.set_cameras([self.cams[view]], self.c_cams[view])
        lut = self.luts[k:k + 1]
        p.project(*P.rendered(), lut, stream)
        if P.lit:
            p.shade(P.mean_v, P.raw[3], P.raw[4], self.lights[view:view + 1], stream)
        p.bin_sort(stream=stream)
        p.composite(lut, self.bg, stream=stream)
        return p.out

    def evaluate(self, pairs, stream=None):
        """Mean (1 - lambda) L1 + lambda (1 - SSIM) over the given (view, map)
        pairs with the current parameters; no gradient or update is kept (the
        pipeline's per-step buffers are overwritten)."""
        p = self.pipe
        vals = torch.empty(len(pairs), device=p.device)
        loss = torch.zeros(3, device=p.device)
        for i, (view, k) in enumerate(pairs):
            self.render(int(view), int(k), stream)
            _lib.veg_l1_ssim_loss(p.out, self.targets[int(view), int(k)], p.loss_grad, loss,
                                  self.loss_ws, self.lam, stream)
            vals[i] = loss[0]
        return float(vals.mean()) if len(pairs) else float("nan")

    def _build_args(self):
        """The native executor's view of every buffer (rebuilt whenever the
        arrays change, i.e. after densification)."""
        p, P, D = self.pipe, self.P, self.density
        p.ensure_shade_buffers()
        ptr = lambda t: None if t is None else t.data_ptr()
        a = _lib.veg_train_args()
        for i in range(5):
            a.raw[i], a.grad[i] = ptr(P.raw[i]), ptr(P.grads[i])
            a.exp_avg[i], a.exp_avg_sq[i] = ptr(P.m[i]), ptr(P.v[i])
        a.mean_v, a.logscale_w, a.n = P.mean_v.data_ptr(), P.logscale_w.data_ptr(), P.n
        if self._c_all is None:
            self._c_all = _lib.cameras(self.cams)
            self._lights_c = np.ascontiguousarray(self.lights, np.float32)
        a.cams, a.n_cams = self._c_all, len(self.cams)
        a.light_dirs = self._lights_c.ctypes.data
        a.luts, a.lut_size, a.n_maps = self.luts.data_ptr(), self.luts.shape[1], self.K
        a.targets = self.targets.data_ptr()
        a.bg[:] = [float(b) for b in self.bg]
        a.lambda_ = self.lam
        a.lr[:] = [float(x) for x in np.asarray(self.lr, np.float64).ravel()]
        a.beta1, a.beta2, a.eps = 0.9, 0.999, 1e-15
        a.lit, a.tf_group = 1 if P.lit else 0, 0
        a.splat_geo, a.splat_aux = p.geo.data_ptr(), p.aux.data_ptr()
        a.tiles_touched, a.rect = p.tiles.data_ptr(), p.rect.data_ptr()
        a.splat_shade, a.grad_shade = p.splat_shade.data_ptr(), p.grad_shade.data_ptr()
        a.binsort_ws, a.binsort_ws_bytes = p.ws.data_ptr(), p.ws.numel()
        a.capacity, a.vals = p.capacity, p.vals.data_ptr()
        a.tile_ranges, a.tile_order = p.ranges.data_ptr(), p.order.data_ptr()
        a.out, a.n_contrib = p.out.data_ptr(), p.n_contrib.data_ptr()
        a.loss_grad, a.grad2d = p.loss_grad.data_ptr(), p.grad2d.data_ptr()
        a.loss, a.loss_ws = self.loss.data_ptr(), self.loss_ws.data_ptr()
        a.loss_ws_bytes = self.loss_ws.numel()
        if D is not None:
            if D.accum is None or D.accum.numel() != P.n:
                D.reset(P.n)
            a.stat_accum, a.stat_count = D.accum.data_ptr(), D.count.data_ptr()
        self._args = a

    def step(self, view=None, k=None, stream=None):
        """One training iteration; returns (view, map) used.  With density
        control, an iteration that densifies replaces the parameter arrays
        instead of taking the Adam step."""
        if view is None:
            view = int(self.rng.integers(len(self.cams)))
        if k is None:
            k = int(self.rng.integers(self.K))
        self.it += 1
        if self.native:
            return self._native_step(view, k, stream)
        p, P, D = self.pipe, self.P, self.density
        self.render(view, k, stream)
        _lib.veg_l1_ssim_loss(p.out, self.targets[view, k], p.loss_grad, self.loss,
                              self.loss_ws, self.lam, stream)
        P.zero_grad()
        p.backward(p.loss_grad, P.grads[0], P.grads[1], P.grads[2], P.grads[3], P.grads[4],
                   stream=stream)
        if D is not None and D.active(self.it):
            D.accumulate(p, P, stream)
        if D is not None and D.due(self.it):
            D.apply(P, stream)
            self.pipe.resize(P.n)
        else:
            P.adam(self.lr, stream)
        return view, k

    def _native_step(self, view, k, stream):
        P, D = self.P, self.density
        if self._args is None:
            self._build_args()
        due = D is not None and D.due(self.it)
        accumulate = D is not None and D.active(self.it)
        _lib.veg_train_step(self._args, view, k, 0 if due else P.step + 1, accumulate, stream)
        if due:
            D.apply(P, stream)
            self.pipe.resize(P.n)
            self._args = None
        else:
            P.step += 1
        return view, k

    def overflowed(self, stream=None):
        """True if the last binning ran out of instance capacity (host sync)."""
        st, _ = self.pipe.status(stream)
        return st != _lib.VEG_OK
