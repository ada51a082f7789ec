"""Device-resident VEG rendering pipeline over the C ABI.

`SplatPipeline` owns the device buffers of one problem shape (n Gaussians,
V views of one size, n_tf transfer functions) and sequences the library's
entry points: veg_project -> veg_bin_sort -> veg_composite_fwd, then
veg_l1_loss and veg_composite_bwd for training.  PyTorch only provides the
memory and the stream; every stage runs in libveg.so.

With Blinn-Phong lighting (Eq. 2-3) `shade` runs veg_shade first; the
compositor then blends s_d C(v) + s_s, and the backward chains the shading
gradients through veg_shade_bwd to the normals, the shininess, the material
coefficients and the means.

`VEGRender` wraps forward/backward as a torch.autograd.Function so that the
sigmoid activations of the stored scalar and weight (Sec. 3.3) and the
optimiser stay in torch.  Its backward reads the pipeline's forward buffers,
so a pipeline serves one render awaiting backward at a time (a second
composite before that backward makes it raise).
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib


def lut_tensor(luts, device="cuda") -> torch.Tensor:
    t = torch.as_tensor(np.asarray(luts, np.float32), device=device)
    return t.reshape(-1, t.shape[-2], 4).contiguous()


def headlight_dirs(cams) -> np.ndarray:
    """[V][3] world directions toward a light on each camera's optical axis,
    behind the camera (the headlight of the paper's reference renders)."""
    return np.stack([-np.asarray(c.world_to_cam, np.float64)[2, :3] for c in cams])


class SplatPipeline:
    """Buffers and stage sequencing for one (n, views, image, n_tf) shape."""

    def __init__(self, n, cams, n_tf, capacity=None, tf_group=0, device="cuda"):
        _lib.load()
        self.n = int(n)
        self.cams = list(cams)
        self.V = len(self.cams)
        self.W, self.H = self.cams[0].width, self.cams[0].height
        self.n_tf = int(n_tf)
        self.tf_group = int(tf_group)      # TFs per compositing pass (forward)
        self.tf_group_bwd = int(tf_group)  # TFs per pass (backward)
        self.tile_batch = 0                # splats staged per pass (forward; 0 = 256)
        self.tile_batch_bwd = 0            # (backward)
        self.device = torch.device(device)
        self.c_cams = _lib.cameras(self.cams)
        nrec = self.V * self.n
        dev = self.device
        self.splat_shade = None
        self.grad_shade = None
        self._shade_rows = None
        self._records(self.n)
        self.tiles_x = (self.W + 15) // 16
        self.tiles_per_view = self.tiles_x * ((self.H + 15) // 16)
        self.ranges = torch.empty(self.V * self.tiles_per_view, 2, dtype=torch.int32, device=dev)
        self.order = torch.empty(self.V * self.tiles_per_view, dtype=torch.int32, device=dev)
        self.out = torch.empty(self.V, self.n_tf, self.H, self.W, 4, device=dev)
        self.n_contrib = torch.empty(self.V, self.n_tf, self.H, self.W, dtype=torch.int32,
                                     device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.loss_grad = torch.empty_like(self.out)
        self.loss_ws = torch.empty(_lib.veg_l1_loss_workspace_size(), dtype=torch.uint8,
                                   device=dev)
        self.keys = None
        self._lit = None  # (mean_v, normal_beta, k_ads, light_dirs) when shaded
        self.generation = 0  # composites so far: a backward must follow its own forward
        self.set_capacity(capacity if capacity is not None else max(1 << 16, 8 * nrec))

    def _records(self, rows):
        """Allocates the per-record buffers for up to `rows` Gaussians per view
        and views their first n."""
        self.rows = int(rows)
        nr, dev = self.V * self.rows, self.device
        self._rec = (torch.empty(nr, 4, device=dev), torch.empty(nr, 4, device=dev),
                     torch.empty(nr, dtype=torch.int32, device=dev),
                     torch.empty(nr, 4, dtype=torch.int16, device=dev),
                     torch.empty(nr * 2, 4, device=dev))
        shaded = self._shade_rows is not None
        self._shade_rows = None
        if shaded:
            self.ensure_shade_buffers()
        self._view_records()

    def _view_records(self):
        nr = self.V * self.n
        geo, aux, tiles, rect, grad2d = self._rec
        self.geo, self.aux, self.tiles, self.rect = geo[:nr], aux[:nr], tiles[:nr], rect[:nr]
        self.grad2d = grad2d[:2 * nr]
        if self._shade_rows is not None:
            self.splat_shade = self._shade_rows[0][:nr]
            self.grad_shade = self._shade_rows[1][:nr]
        else:
            self.splat_shade = self.grad_shade = None

    def ensure_shade_buffers(self):
        """Per-(view, Gaussian) Blinn-Phong factors and their gradients."""
        if self._shade_rows is None:
            nr = self.V * self.rows
            self._shade_rows = (torch.empty(nr, 2, device=self.device),
                                torch.empty(nr, 2, device=self.device))
            self._view_records()

    def resize(self, n):
        """Adapts the pipeline to n Gaussians per view (after densification):
        the buffers stay when n fits the allocated rows (the binning status
        is kept), else they are reallocated with 25% headroom and the
        binning workspace starts afresh (no binning yet)."""
        n = int(n)
        self.n = n
        if n > self.rows:
            self._records(n + n // 4)
            self.set_capacity(self.capacity)
        else:
            self._view_records()

    def set_cameras(self, cams, c_cams=None):
        """Switch to other cameras of the same count and image size (c_cams:
        their prebuilt C structs, optional)."""
        cams = list(cams)
        if len(cams) != self.V or cams[0].width != self.W or cams[0].height != self.H:
            raise ValueError("set_cameras needs the same number of views and image size")
        self.cams = cams
        self.c_cams = c_cams if c_cams is not None else _lib.cameras(cams)

    def set_capacity(self, capacity):
        self.capacity = int(capacity)
        ws = _lib.veg_bin_sort_workspace_size(self.rows, self.V, self.capacity, self.W, self.H)
        self.ws = torch.empty(ws, dtype=torch.uint8, device=self.device)
        self.ws[:256].zero_()  # status header: no binning yet, no overflow
        self.vals = torch.empty(max(self.capacity, 1), dtype=torch.int32, device=self.device)

    # -- stages ------------------------------------------------------------
    def project(self, mean_v, logscale_w, quat, cull_luts=None, stream=None):
        self._g = _lib.gaussians(mean_v, logscale_w, quat)
        self._gt = (mean_v, logscale_w, quat)
        tf = _lib.tf_desc(cull_luts) if cull_luts is not None else None
        _lib.veg_project(self.c_cams, self._g, tf, self.geo, self.aux, self.tiles, self.rect,
                         stream)

    def shade(self, mean_v, normal_beta, k_ads, light_dirs, stream=None):
        """Blinn-Phong factors of every view (veg_shade); later composites and
        backward passes are shaded until `unshade`."""
        self.ensure_shade_buffers()
        light_dirs = np.asarray(light_dirs, np.float32).reshape(self.V, 3)
        self._lit = (mean_v, normal_beta, k_ads, light_dirs)
        _lib.veg_shade(self.c_cams, mean_v, normal_beta, k_ads, light_dirs, self.splat_shade,
                       stream)

    def unshade(self):
        self._lit = None

    def bin_sort(self, want_keys=False, stream=None):
        keys = None
        if want_keys:
            if self.keys is None or self.keys.numel() < self.capacity:
                self.keys = torch.empty(max(self.capacity, 1), dtype=torch.int64,
                                        device=self.device)
            keys = self.keys
        _lib.veg_bin_sort(self.c_cams, self.n, self.geo, self.tiles, self.rect, self.ws,
                          self.capacity, keys, self.vals, self.ranges, stream)
        _lib.veg_tile_order(self.ranges, self.order, stream)

    def status(self, stream=None):
        """(status, instance count) after waiting for the stream; raises if a
        bounded device-side wait of the binning gave up (its lists are void)."""
        st, m = _lib.veg_sync_status(self.ws, stream)
        if st == _lib.VEG_ERR_TIMEOUT:
            raise _lib.VegError("veg_bin_sort", st)
        return st, m

    def composite(self, luts, bg=(0.0, 0.0, 0.0), stats=None, stream=None):
        self.generation += 1
        self._luts = luts
        self._bg = tuple(float(b) for b in bg)
        _lib.veg_composite_fwd(self.c_cams, self.n, self.geo, self.aux, self.vals, self.ranges,
                               _lib.tf_desc(luts), self._bg, self.tf_group, self.out,
                               self.n_contrib, stats, stream, tile_order=self.order,
                               splat_shade=self._shade_buf(), tile_batch=self.tile_batch)
        return self.out

    def _shade_buf(self):
        return self.splat_shade if self._lit is not None else None

    def _grad_shade_buf(self):
        return self.grad_shade if self._lit is not None else None

    def l1(self, target, stream=None):
        _lib.veg_l1_loss(self.out, target, self.out.numel() // 4, self.loss_grad, self.loss,
                         self.loss_ws, stream)
        return self.loss

    def backward(self, dL_dout, grad_mean_v, grad_logscale_w, grad_quat, grad_normal_beta=None,
                 grad_k_ads=None, stream=None):
        """Accumulates the gradients of every parameter; when shaded, also
        those of the lighting parameters (grad_normal_beta, grad_k_ads)."""
        _lib.veg_composite_bwd(self.c_cams, self._g, self.geo, self.aux, self.tiles, self.vals,
                               self.ranges, _lib.tf_desc(self._luts), self._bg,
                               self.tf_group_bwd,
                               self.out, self.n_contrib, dL_dout, None, grad_mean_v,
                               grad_logscale_w, grad_quat, self.grad2d, None, stream,
                               tile_order=self.order, splat_shade=self._shade_buf(),
                               grad_shade=self._grad_shade_buf(), tile_batch=self.tile_batch_bwd)
        if self._lit is not None:
            self.shade_backward(grad_mean_v, grad_normal_beta, grad_k_ads, stream)

    def backward_2d(self, dL_dout, stats=None, stream=None):
        """Screen-space gradients only (into self.grad2d, and self.grad_shade
        when shaded)."""
        _lib.veg_composite_bwd(self.c_cams, self._g, self.geo, self.aux, self.tiles, self.vals,
                               self.ranges, _lib.tf_desc(self._luts), self._bg,
                               self.tf_group_bwd,
                               self.out, self.n_contrib, dL_dout, None, None, None, None,
                               self.grad2d, stats, stream, tile_order=self.order,
                               splat_shade=self._shade_buf(), grad_shade=self._grad_shade_buf(),
                               tile_batch=self.tile_batch_bwd)

    def project_backward(self, grad_mean_v, grad_logscale_w, grad_quat, stream=None,
                         first=0, count=None):
        """Accumulates the projection backward of Gaussians [first, first +
        count) (all by default) from self.grad2d into the gradients."""
        if first == 0 and count is None:
            _lib.veg_project_bwd(self.c_cams, self._g, self.tiles, self.grad2d, grad_mean_v,
                                 grad_logscale_w, grad_quat, stream)
            return
        count = self.n - first if count is None else count
        _lib.veg_project_bwd_range(self.c_cams, self._g, self.tiles, self.grad2d, first, count,
                                   grad_mean_v, grad_logscale_w, grad_quat, stream)

    def shade_backward(self, grad_mean_v, grad_normal_beta, grad_k_ads, stream=None):
        if grad_normal_beta is None or grad_k_ads is None:
            raise ValueError("a shaded backward needs grad_normal_beta and grad_k_ads")
        mean_v, normal_beta, k_ads, light_dirs = self._lit
        _lib.veg_shade_bwd(self.c_cams, mean_v, normal_beta, k_ads, light_dirs, self.tiles,
                           self.grad_shade, grad_mean_v, grad_normal_beta, grad_k_ads, stream)

    # -- whole passes --------------------------------------------------------
    def render(self, mean_v, logscale_w, quat, luts, bg=(0.0, 0.0, 0.0), cull=True,
               stream=None):
        """Project + bin + composite; grows the instance capacity (one host
        sync) when the binning overflowed."""
        self.project(mean_v, logscale_w, quat, luts if cull else None, stream)
        self.bin_sort(stream=stream)
        st, m = self.status(stream)
        if st != _lib.VEG_OK:
            self.set_capacity(int(m * 1.25) + 1024)
            self.bin_sort(stream=stream)
        return self.composite(luts, bg, stream=stream)

    def train_step(self, mean_v, logscale_w, quat, luts, target, grads, bg=(0.0, 0.0, 0.0),
                   lighting=None, stream=None, project_grads=True):
        """One pass of the hot path: project, bin, sort, (shade,) composite,
        L1 loss, composite backward, projection (and shading) backward.
        grads = (mean_v, logscale_w, quat[, normal_beta, k_ads]) gradient
        buffers, zeroed first; lighting = (normal_beta, k_ads, light_dirs).
        With project_grads=False the projection backward is left to the
        caller (e.g. a bucketed one overlapping the gradient all-reduce)."""
        for gbuf in grads:
            gbuf.zero_()
        self.project(mean_v, logscale_w, quat, luts, stream)
        if lighting is not None:
            self.shade(mean_v, *lighting, stream=stream)
        else:
            self.unshade()
        self.bin_sort(stream=stream)
        self.composite(luts, bg, stream=stream)
        self.l1(target, stream)
        if project_grads:
            self.backward(self.loss_grad, *grads, stream=stream)
        else:
            self.backward_2d(self.loss_grad, stream=stream)
            if self._lit is not None:
                self.shade_backward(grads[0], grads[3], grads[4], stream)
        return self.loss


class VEGRender(torch.autograd.Function):
    """out[V,T,H,W,4] = render(mean_v, logscale_w, quat[, normal_beta, k_ads])
    for fixed cameras, transfer functions, background (and light
    directions); gradients from veg_composite_bwd (and veg_shade_bwd)."""

    @staticmethod
    def forward(ctx, mean_v, logscale_w, quat, normal_beta, k_ads, pipeline: SplatPipeline, luts,
                bg, light_dirs):
        mean_v, logscale_w, quat = (t.contiguous() for t in (mean_v, logscale_w, quat))
        lit = normal_beta is not None
        pipeline.project(mean_v, logscale_w, quat, luts)
        if lit:
            normal_beta, k_ads = normal_beta.contiguous(), k_ads.contiguous()
            pipeline.shade(mean_v, normal_beta, k_ads, light_dirs)
        else:
            pipeline.unshade()
        pipeline.bin_sort()
        st, m = pipeline.status()
        if st != _lib.VEG_OK:
            pipeline.set_capacity(int(m * 1.25) + 1024)
            pipeline.bin_sort()
        out = pipeline.composite(luts, bg)
        ctx.pipeline = pipeline
        ctx.generation = pipeline.generation
        ctx.lit = lit
        if lit:
            ctx.save_for_backward(mean_v, logscale_w, quat, normal_beta, k_ads)
        else:
            ctx.save_for_backward(mean_v, logscale_w, quat)
        return out.clone()

    @staticmethod
    def backward(ctx, dout):
        saved = ctx.saved_tensors
        p = ctx.pipeline
        if p.generation != ctx.generation:
            raise RuntimeError("the pipeline composited again after this render: its buffers no "
                               "longer hold it (use one pipeline per render awaiting backward)")
        gm, gl, gq = (torch.zeros_like(t) for t in saved[:3])
        if ctx.lit:
            gn = torch.zeros_like(saved[3])
            gk = torch.zeros_like(saved[4])
            p.backward(dout.contiguous(), gm, gl, gq, gn, gk)
            return gm, gl, gq, gn, gk, None, None, None, None
        p.backward(dout.contiguous(), gm, gl, gq)
        return gm, gl, gq, None, None, None, None, None, None


def render(mean_v, logscale_w, quat, pipeline, luts, bg=(0.0, 0.0, 0.0), normal_beta=None,
           k_ads=None, light_dirs=None):
    """Differentiable render; Blinn-Phong shaded when normal_beta [n][4]
    (normal, beta), k_ads [n][4] (k_a, k_d, k_s, -) and light_dirs [V][3]
    are given."""
    return VEGRender.apply(mean_v, logscale_w, quat, normal_beta, k_ads, pipeline, luts, bg,
                           light_dirs)
