"""Device-resident VEG rendering pipeline over the C ABI.

`SplatPipeline` owns the device buffers of one problem shape (n Gaussians,
V views of one size, n_tf transfer functions) and sequences the library's
entry points: veg_project -> veg_bin_sort -> veg_composite_fwd, then
veg_l1_loss and veg_composite_bwd for training.  PyTorch only provides the
memory and the stream; every stage runs in libveg.so.

`VEGRender` wraps forward/backward as a torch.autograd.Function so that the
sigmoid activations of the stored scalar and weight (Sec. 3.3) and the
optimiser stay in torch.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib


def lut_tensor(luts, device="cuda") -> torch.Tensor:
    t = torch.as_tensor(np.asarray(luts, np.float32), device=device)
    return t.reshape(-1, t.shape[-2], 4).contiguous()


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
        self.device = torch.device(device)
        self.c_cams = _lib.cameras(self.cams)
        nrec = self.V * self.n
        dev = self.device
        self.geo = torch.empty(nrec, 4, device=dev)
        self.aux = torch.empty(nrec, 4, device=dev)
        self.tiles = torch.empty(nrec, dtype=torch.int32, device=dev)
        self.rect = torch.empty(nrec, 4, dtype=torch.int16, device=dev)
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
        self.grad2d = torch.empty(nrec * 2, 4, device=dev)
        self.keys = None
        self.set_capacity(capacity if capacity is not None else max(1 << 16, 8 * nrec))

    def set_capacity(self, capacity):
        self.capacity = int(capacity)
        ws = _lib.veg_bin_sort_workspace_size(self.n, self.V, self.capacity, self.W, self.H)
        self.ws = torch.empty(ws, dtype=torch.uint8, device=self.device)
        self.vals = torch.empty(max(self.capacity, 1), dtype=torch.int32, device=self.device)

    # -- stages ------------------------------------------------------------
    def project(self, mean_v, logscale_w, quat, cull_luts=None, stream=None):
        self._g = _lib.gaussians(mean_v, logscale_w, quat)
        self._gt = (mean_v, logscale_w, quat)
        tf = _lib.tf_desc(cull_luts) if cull_luts is not None else None
        _lib.veg_project(self.c_cams, self._g, tf, self.geo, self.aux, self.tiles, self.rect,
                         stream)

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
        """(status, instance count) after waiting for the stream."""
        return _lib.veg_sync_status(self.ws, stream)

    def composite(self, luts, bg=(0.0, 0.0, 0.0), stats=None, stream=None):
        self._luts = luts
        self._bg = tuple(float(b) for b in bg)
        _lib.veg_composite_fwd(self.c_cams, self.n, self.geo, self.aux, self.vals, self.ranges,
                               _lib.tf_desc(luts), self._bg, self.tf_group, self.out,
                               self.n_contrib, stats, stream, tile_order=self.order)
        return self.out

    def l1(self, target, stream=None):
        _lib.veg_l1_loss(self.out, target, self.out.numel() // 4, self.loss_grad, self.loss,
                         self.loss_ws, stream)
        return self.loss

    def backward(self, dL_dout, grad_mean_v, grad_logscale_w, grad_quat, stream=None):
        _lib.veg_composite_bwd(self.c_cams, self._g, self.geo, self.aux, self.tiles, self.vals,
                               self.ranges, _lib.tf_desc(self._luts), self._bg,
                               self.tf_group_bwd,
                               self.out, self.n_contrib, dL_dout, None, grad_mean_v,
                               grad_logscale_w, grad_quat, self.grad2d, None, stream,
                               tile_order=self.order)

    def backward_2d(self, dL_dout, stats=None, stream=None):
        """Screen-space gradients only (into self.grad2d)."""
        _lib.veg_composite_bwd(self.c_cams, self._g, self.geo, self.aux, self.tiles, self.vals,
                               self.ranges, _lib.tf_desc(self._luts), self._bg,
                               self.tf_group_bwd,
                               self.out, self.n_contrib, dL_dout, None, None, None, None,
                               self.grad2d, stats, stream, tile_order=self.order)

    def project_backward(self, grad_mean_v, grad_logscale_w, grad_quat, stream=None):
        _lib.veg_project_bwd(self.c_cams, self._g, self.tiles, self.grad2d, grad_mean_v,
                             grad_logscale_w, grad_quat, stream)

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
                   stream=None):
        """One pass of the hot path: project, bin, sort, composite, L1 loss,
        composite backward, projection backward (grads are zeroed first)."""
        for gbuf in grads:
            gbuf.zero_()
        self.project(mean_v, logscale_w, quat, luts, stream)
        self.bin_sort(stream=stream)
        self.composite(luts, bg, stream=stream)
        self.l1(target, stream)
        self.backward(self.loss_grad, *grads, stream=stream)
        return self.loss


class VEGRender(torch.autograd.Function):
    """out[V,T,H,W,4] = render(mean_v, logscale_w, quat) for fixed cameras,
    transfer functions and background; gradients from veg_composite_bwd."""

    @staticmethod
    def forward(ctx, mean_v, logscale_w, quat, pipeline: SplatPipeline, luts, bg):
        mean_v, logscale_w, quat = (t.contiguous() for t in (mean_v, logscale_w, quat))
        out = pipeline.render(mean_v, logscale_w, quat, luts, bg)
        ctx.pipeline = pipeline
        ctx.save_for_backward(mean_v, logscale_w, quat)
        return out.clone()

    @staticmethod
    def backward(ctx, dout):
        mean_v, logscale_w, quat = ctx.saved_tensors
        p = ctx.pipeline
        gm = torch.zeros_like(mean_v)
        gl = torch.zeros_like(logscale_w)
        gq = torch.zeros_like(quat)
        p.backward(dout.contiguous(), gm, gl, gq)
        return gm, gl, gq, None, None, None


def render(mean_v, logscale_w, quat, pipeline, luts, bg=(0.0, 0.0, 0.0)):
    return VEGRender.apply(mean_v, logscale_w, quat, pipeline, luts, bg)
