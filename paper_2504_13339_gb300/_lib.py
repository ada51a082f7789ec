"""ctypes binding of libveg.so: argument marshalling only.

Every function here has the name of the C entry point it calls and takes
torch CUDA tensors (device memory) plus plain numbers; nothing is computed in
Python.  Importing this module fails loudly if the library has not been built:
there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libveg.so")

VEG_OK = 0
VEG_MAX_VIEWS = 64  # include/veg.h
VEG_ERR_CAPACITY = 2
VEG_ERR_TIMEOUT = 4
STATUS_NAMES = {0: "VEG_OK", 1: "VEG_ERR_INVALID_ARGUMENT", 2: "VEG_ERR_CAPACITY",
                3: "VEG_ERR_CUDA", 4: "VEG_ERR_TIMEOUT", 5: "VEG_ERR_UNSUPPORTED"}
MAX_VIEWS = 64


class VegError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        super().__init__(f"{fn} failed: {STATUS_NAMES.get(status, status)}")


class veg_camera(ctypes.Structure):
    _fields_ = [("world_to_cam", ctypes.c_float * 12), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("near_plane", ctypes.c_float)]


class veg_gaussians(ctypes.Structure):
    _fields_ = [("mean_v", ctypes.c_void_p), ("logscale_w", ctypes.c_void_p),
                ("quat", ctypes.c_void_p), ("n", ctypes.c_int64)]


class veg_tf(ctypes.Structure):
    _fields_ = [("lut", ctypes.c_void_p), ("lut_size", ctypes.c_int32), ("n_tf", ctypes.c_int32),
                ("view_tf", ctypes.c_void_p)]


class veg_adam_arrays(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p * 5), ("grad", ctypes.c_void_p * 5),
                ("exp_avg", ctypes.c_void_p * 5), ("exp_avg_sq", ctypes.c_void_p * 5),
                ("rendered", ctypes.c_void_p * 2)]


class veg_density_config(ctypes.Structure):
    _fields_ = [("grad_threshold", ctypes.c_float), ("log_size_threshold", ctypes.c_float),
                ("raw_weight_threshold", ctypes.c_float), ("log_split_factor", ctypes.c_float)]


class veg_material(ctypes.Structure):
    _fields_ = [("ka", ctypes.c_float), ("kd", ctypes.c_float), ("ks", ctypes.c_float),
                ("beta", ctypes.c_float)]


_VP = ctypes.c_void_p


class veg_train_args(ctypes.Structure):
    _fields_ = [("raw", _VP * 5), ("grad", _VP * 5), ("exp_avg", _VP * 5),
                ("exp_avg_sq", _VP * 5), ("mean_v", _VP), ("logscale_w", _VP),
                ("n", ctypes.c_int64), ("cams", ctypes.POINTER(veg_camera)),
                ("n_cams", ctypes.c_int32), ("light_dirs", _VP), ("luts", _VP),
                ("lut_size", ctypes.c_int32), ("n_maps", ctypes.c_int32), ("targets", _VP),
                ("bg", ctypes.c_float * 3), ("lambda_", ctypes.c_float),
                ("lr", ctypes.c_float * 20), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("lit", ctypes.c_int32),
                ("tf_group", ctypes.c_int32), ("splat_geo", _VP), ("splat_aux", _VP),
                ("tiles_touched", _VP), ("rect", _VP), ("splat_shade", _VP),
                ("grad_shade", _VP), ("binsort_ws", _VP), ("binsort_ws_bytes", ctypes.c_size_t),
                ("capacity", ctypes.c_int64), ("vals", _VP), ("tile_ranges", _VP),
                ("tile_order", _VP), ("out", _VP), ("n_contrib", _VP), ("loss_grad", _VP),
                ("grad2d", _VP), ("loss", _VP), ("loss_ws", _VP),
                ("loss_ws_bytes", ctypes.c_size_t), ("stat_accum", _VP), ("stat_count", _VP)]


_P = ctypes.c_void_p
_I32, _I64, _SZ = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
_CAMS = ctypes.POINTER(veg_camera)
_SIGS = {
    "veg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "veg_kernel_launches": (ctypes.c_uint64, []),
    "veg_project": (ctypes.c_int, [_CAMS, _I32, veg_gaussians, ctypes.POINTER(veg_tf), _P, _P, _P,
                                   _P, _P]),
    "veg_bin_sort_workspace_size": (ctypes.c_int, [_I64, _I32, _I64, _I32, _I32,
                                                   ctypes.POINTER(_SZ)]),
    "veg_bin_sort": (ctypes.c_int, [_CAMS, _I32, _I64, _P, _P, _P, _P, _SZ, _I64, _P, _P, _P, _P]),
    "veg_bin_sort_static": (ctypes.c_int, [_CAMS, _I32, _I64, _P, _P, _P, _I64, _P, _P, _P, _P,
                                           _P]),
    "veg_sync_status": (ctypes.c_int, [_P, _P, ctypes.POINTER(_I64)]),
    "veg_composite_fwd": (ctypes.c_int, [_CAMS, _I32, _I64, _P, _P, _P, _P, _P, _P, veg_tf, _P,
                                         _I32, _I32, _P, _P, _P, _P]),
    "veg_composite_bwd_workspace_size": (ctypes.c_int, [_I64, _I32, ctypes.POINTER(_SZ)]),
    "veg_composite_bwd": (ctypes.c_int, [_CAMS, _I32, veg_gaussians, _P, _P, _P, _P, _P, _P, _P,
                                         veg_tf, _P, _I32, _I32, _P, _P, _P, _P, _SZ, _P, _P, _P,
                                         _P, _P, _P, _P]),
    "veg_tile_order": (ctypes.c_int, [_P, _I64, _P, _P]),
    "veg_radix_lookback_check": (ctypes.c_int, [_P, _SZ, _I64, _I32, _I32, _P, _P, _P]),
    "veg_project_bwd": (ctypes.c_int, [_CAMS, _I32, veg_gaussians, _P, _P, _P, _P, _P, _P]),
    "veg_project_views": (ctypes.c_int, [_CAMS, _I32, ctypes.POINTER(veg_gaussians), _I64,
                                         ctypes.POINTER(veg_tf), _P, _P, _P, _P, _P]),
    "veg_project_bwd_range": (ctypes.c_int, [_CAMS, _I32, veg_gaussians, _P, _P, _I64, _I64, _P,
                                             _P, _P, _P]),
    "veg_l1_loss_workspace_size": (ctypes.c_int, [ctypes.POINTER(_SZ)]),
    "veg_l1_loss": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P, _SZ, _P]),
    "veg_render_workspace_size": (ctypes.c_int, [_I64, _I32, _I64, _I32, _I32,
                                                 ctypes.POINTER(_SZ)]),
    "veg_render": (ctypes.c_int, [_CAMS, _I32, veg_gaussians, veg_tf, _P, _I32, _I64, _P, _SZ, _P,
                                  _P, _P]),
    "veg_shade": (ctypes.c_int, [_CAMS, _I32, _P, _I64, _P, _P, _P, _P, _P]),
    "veg_l1_ssim_loss_workspace_size": (ctypes.c_int, [_I64, _I32, _I32, ctypes.POINTER(_SZ)]),
    "veg_l1_ssim_loss": (ctypes.c_int, [_P, _P, _I64, _I32, _I32, ctypes.c_float, _P, _P, _P, _SZ,
                                        _P]),
    "veg_adam_step": (ctypes.c_int, [ctypes.POINTER(veg_adam_arrays), _I64, _P, ctypes.c_float,
                                     ctypes.c_float, ctypes.c_float, _I32, _P]),
    "veg_adam_step_counted": (ctypes.c_int, [ctypes.POINTER(veg_adam_arrays), _I64, _P,
                                             ctypes.c_float, ctypes.c_float, ctypes.c_float, _P,
                                             _P]),
    "veg_volume_prepare": (ctypes.c_int, [_P, _I32, _P, _P]),
    "veg_train_step": (ctypes.c_int, [ctypes.POINTER(veg_train_args), _I32, _I32, _I32, _I32,
                                      _P]),
    "veg_raymarch": (ctypes.c_int, [_CAMS, _I32, _P, _I32, veg_tf, ctypes.c_float,
                                    ctypes.POINTER(veg_material), _P, _P, _P, _P]),
    "veg_raymarch_cells_count": (ctypes.c_int, [_I32, _I32, ctypes.POINTER(ctypes.c_int64)]),
    "veg_raymarch_cells": (ctypes.c_int, [_P, _I32, veg_tf, _I32, _P, _P]),
    "veg_raymarch_masked": (ctypes.c_int, [_CAMS, _I32, _P, _I32, veg_tf, ctypes.c_float,
                                           ctypes.POINTER(veg_material), _P, _P, _I32, _P, _P,
                                           _P]),
    "veg_grad_stats_accumulate": (ctypes.c_int, [_P, _P, _I64, _I32, _I32, _I32, _P, _P, _P]),
    "veg_densify_workspace_size": (ctypes.c_int, [_I64, ctypes.POINTER(_SZ)]),
    "veg_densify": (ctypes.c_int, [ctypes.POINTER(veg_adam_arrays), _I64, _P, _P, _P,
                                   veg_density_config, ctypes.POINTER(veg_adam_arrays), _I64, _P,
                                   _P, _P, _SZ, _P]),
    "veg_shade_bwd": (ctypes.c_int, [_CAMS, _I32, _P, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
}
EXPORTED = tuple(_SIGS)

_lib = None


def load(path: str = LIB_PATH):
    """Loads libveg.so (raises if it is missing) and declares every symbol."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libveg.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(name, status):
    if status != VEG_OK:
        raise VegError(name, status)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def cameras(cams):
    """ctypes array of veg_camera from scene cameras."""
    arr = (veg_camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i].world_to_cam[:] = [float(x) for x in np.asarray(c.world_to_cam, np.float32).ravel()]
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = c.fx, c.fy, c.cx, c.cy
        arr[i].width, arr[i].height, arr[i].near_plane = c.width, c.height, c.near
    return arr


def gaussians(mean_v, logscale_w, quat):
    return veg_gaussians(mean_v.data_ptr(), logscale_w.data_ptr(), quat.data_ptr(),
                         mean_v.shape[0])


def tf_desc(luts, view_tf=None):
    """Descriptor of TF tables luts [n_tf][L][4]; view_tf (device int32 [V])
    selects one table per view."""
    return veg_tf(luts.data_ptr(), luts.shape[-2], luts.shape[0],
                  None if view_tf is None else view_tf.data_ptr())


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def veg_status_string(status: int) -> str:
    return load().veg_status_string(status).decode()


def veg_kernel_launches() -> int:
    return int(load().veg_kernel_launches())


def veg_project(cams, g, cull_tf, splat_geo, splat_aux, tiles_touched, rect, stream=None):
    lib = load()
    tf = ctypes.byref(cull_tf) if cull_tf is not None else None
    _check("veg_project", lib.veg_project(cams, len(cams), g, tf, _ptr(splat_geo), _ptr(splat_aux),
                                          _ptr(tiles_touched), _ptr(rect), _stream(stream)))


def veg_project_views(cams, models, n, cull_tf, splat_geo, splat_aux, tiles_touched, rect,
                      stream=None):
    """models: one veg_gaussians per view (len(cams) of them); n: the record
    stride (>= every model's n)."""
    lib = load()
    arr = (veg_gaussians * len(models))(*models)
    tf = ctypes.byref(cull_tf) if cull_tf is not None else None
    _check("veg_project_views",
           lib.veg_project_views(cams, len(cams), arr, int(n), tf, _ptr(splat_geo),
                                 _ptr(splat_aux), _ptr(tiles_touched), _ptr(rect),
                                 _stream(stream)))


def veg_bin_sort_workspace_size(n, n_views, capacity, width, height) -> int:
    out = _SZ()
    _check("veg_bin_sort_workspace_size",
           load().veg_bin_sort_workspace_size(n, n_views, capacity, width, height,
                                              ctypes.byref(out)))
    return out.value


def veg_bin_sort(cams, n, splat_geo, tiles_touched, rect, workspace, capacity, keys, vals,
                 tile_ranges, stream=None):
    _check("veg_bin_sort",
           load().veg_bin_sort(cams, len(cams), n, _ptr(splat_geo), _ptr(tiles_touched),
                               _ptr(rect), _ptr(workspace), workspace.numel(), capacity,
                               _ptr(keys), _ptr(vals), _ptr(tile_ranges), _stream(stream)))


def veg_bin_sort_static(cams, n, splat_geo, tiles_touched, rect, capacity, keys, vals,
                        tile_ranges, n_instances, stream=None):
    """veg_bin_sort with the library's fixed device scratch (no workspace);
    returns the raw status so callers can see VEG_ERR_UNSUPPORTED."""
    return load().veg_bin_sort_static(cams, len(cams), n, _ptr(splat_geo), _ptr(tiles_touched),
                                      _ptr(rect), capacity, _ptr(keys), _ptr(vals),
                                      _ptr(tile_ranges), _ptr(n_instances), _stream(stream))


def veg_radix_lookback_check(workspace, n, starve_first, spins, keys_out, vals_out,
                             stream=None):
    _check("veg_radix_lookback_check",
           load().veg_radix_lookback_check(_ptr(workspace), workspace.numel(), n,
                                           int(bool(starve_first)), spins, _ptr(keys_out),
                                           _ptr(vals_out), _stream(stream)))


def veg_sync_status(workspace, stream=None):
    """Returns (status, n_instances); does not raise on VEG_ERR_CAPACITY or
    VEG_ERR_TIMEOUT (the caller decides)."""
    n = _I64()
    st = load().veg_sync_status(_ptr(workspace), _stream(stream), ctypes.byref(n))
    if st not in (VEG_OK, VEG_ERR_CAPACITY, VEG_ERR_TIMEOUT):
        raise VegError("veg_sync_status", st)
    return st, n.value


def veg_tile_order(tile_ranges, tile_order, stream=None):
    _check("veg_tile_order", load().veg_tile_order(_ptr(tile_ranges), tile_ranges.shape[0],
                                                   _ptr(tile_order), _stream(stream)))


def veg_composite_fwd(cams, n, splat_geo, splat_aux, vals, tile_ranges, tf, bg, tf_group, out,
                      n_contrib, stats=None, stream=None, tile_order=None, splat_shade=None,
                      tile_batch=0):
    bgc = (ctypes.c_float * 3)(*[float(b) for b in bg])
    _check("veg_composite_fwd",
           load().veg_composite_fwd(cams, len(cams), n, _ptr(splat_geo), _ptr(splat_aux),
                                    _ptr(splat_shade), _ptr(vals), _ptr(tile_ranges), _ptr(tile_order), tf,
                                    ctypes.cast(bgc, ctypes.c_void_p), tf_group, tile_batch,
                                    _ptr(out), _ptr(n_contrib), _ptr(stats), _stream(stream)))


def veg_composite_bwd_workspace_size(n, n_views) -> int:
    out = _SZ()
    _check("veg_composite_bwd_workspace_size",
           load().veg_composite_bwd_workspace_size(n, n_views, ctypes.byref(out)))
    return out.value


def veg_composite_bwd(cams, g, splat_geo, splat_aux, tiles_touched, vals, tile_ranges, tf, bg,
                      tf_group, out, n_contrib, dL_dout, workspace, grad_mean_v, grad_logscale_w,
                      grad_quat, grad2d=None, stats=None, stream=None, tile_order=None,
                      splat_shade=None, grad_shade=None, tile_batch=0):
    bgc = (ctypes.c_float * 3)(*[float(b) for b in bg])
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check("veg_composite_bwd",
           load().veg_composite_bwd(cams, len(cams), g, _ptr(splat_geo), _ptr(splat_aux),
                                    _ptr(splat_shade), _ptr(tiles_touched), _ptr(vals), _ptr(tile_ranges),
                                    _ptr(tile_order), tf,
                                    ctypes.cast(bgc, ctypes.c_void_p), tf_group, tile_batch,
                                    _ptr(out), _ptr(n_contrib), _ptr(dL_dout), _ptr(workspace),
                                    ws_bytes,
                                    _ptr(grad_mean_v), _ptr(grad_logscale_w), _ptr(grad_quat),
                                    _ptr(grad2d), _ptr(grad_shade), _ptr(stats),
                                    _stream(stream)))


def _lights(light_dirs):
    l = np.ascontiguousarray(np.asarray(light_dirs, np.float32).reshape(-1, 3))
    return l, ctypes.c_void_p(l.ctypes.data)


def veg_shade(cams, mean_v, normal_beta, k_ads, light_dirs, splat_shade, stream=None):
    """Blinn-Phong factors (s_d, s_s) per view and Gaussian; light_dirs is a
    host array [V][3]."""
    keep, lp = _lights(light_dirs)
    _check("veg_shade",
           load().veg_shade(cams, len(cams), _ptr(mean_v), mean_v.shape[0], _ptr(normal_beta),
                            _ptr(k_ads), lp, _ptr(splat_shade), _stream(stream)))
    del keep


def veg_shade_bwd(cams, mean_v, normal_beta, k_ads, light_dirs, tiles_touched, grad_shade,
                  grad_mean_v, grad_normal_beta, grad_k_ads, stream=None):
    keep, lp = _lights(light_dirs)
    _check("veg_shade_bwd",
           load().veg_shade_bwd(cams, len(cams), _ptr(mean_v), mean_v.shape[0],
                                _ptr(normal_beta), _ptr(k_ads), lp, _ptr(tiles_touched),
                                _ptr(grad_shade), _ptr(grad_mean_v), _ptr(grad_normal_beta),
                                _ptr(grad_k_ads), _stream(stream)))
    del keep


def veg_l1_ssim_loss_workspace_size(n_images, height, width) -> int:
    out = _SZ()
    _check("veg_l1_ssim_loss_workspace_size",
           load().veg_l1_ssim_loss_workspace_size(n_images, height, width, ctypes.byref(out)))
    return out.value


def veg_l1_ssim_loss(out, target, grad, loss, workspace, lam=0.2, stream=None):
    """out/target/grad [..., H, W, 4]; loss: device float[3]."""
    H, W = out.shape[-3], out.shape[-2]
    n_img = out.numel() // (H * W * 4)
    _check("veg_l1_ssim_loss",
           load().veg_l1_ssim_loss(_ptr(out), _ptr(target), n_img, H, W, float(lam), _ptr(grad),
                                   _ptr(loss), _ptr(workspace),
                                   workspace.numel() * workspace.element_size(),
                                   _stream(stream)))


def adam_arrays(params, grads, exp_avg, exp_avg_sq, rendered=(None, None)):
    """veg_adam_arrays from five-element lists of tensors (or None)."""
    a = veg_adam_arrays()
    for i in range(5):
        a.param[i] = None if params[i] is None else params[i].data_ptr()
        a.grad[i] = None if grads[i] is None else grads[i].data_ptr()
        a.exp_avg[i] = None if exp_avg[i] is None else exp_avg[i].data_ptr()
        a.exp_avg_sq[i] = None if exp_avg_sq[i] is None else exp_avg_sq[i].data_ptr()
    for i in range(2):
        a.rendered[i] = None if rendered[i] is None else rendered[i].data_ptr()
    return a


def veg_adam_step(arrays, n, lr, step, beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
    lrs = (ctypes.c_float * 20)(*[float(x) for x in np.asarray(lr, np.float64).ravel()])
    _check("veg_adam_step",
           load().veg_adam_step(ctypes.byref(arrays), n, ctypes.cast(lrs, ctypes.c_void_p),
                                beta1, beta2, eps, step, _stream(stream)))


def veg_adam_step_counted(arrays, n, lr, counter, beta1=0.9, beta2=0.999, eps=1e-15,
                          stream=None):
    """counter: 16-byte device tensor (e.g. torch.zeros(2, dtype=torch.int64)) holding the
    steps taken, zeroed before the first step; advanced by one on the device."""
    lrs = (ctypes.c_float * 20)(*[float(x) for x in np.asarray(lr, np.float64).ravel()])
    _check("veg_adam_step_counted",
           load().veg_adam_step_counted(ctypes.byref(arrays), n, ctypes.cast(lrs, ctypes.c_void_p),
                                        beta1, beta2, eps, _ptr(counter), _stream(stream)))


def veg_grad_stats_accumulate(grad2d, tiles_touched, n, n_views, width, height, accum, count,
                              stream=None):
    _check("veg_grad_stats_accumulate",
           load().veg_grad_stats_accumulate(_ptr(grad2d), _ptr(tiles_touched), n, n_views, width,
                                            height, _ptr(accum), _ptr(count), _stream(stream)))


def veg_densify_workspace_size(n) -> int:
    out = _SZ()
    _check("veg_densify_workspace_size", load().veg_densify_workspace_size(n, ctypes.byref(out)))
    return out.value


def veg_densify(in_arrays, n, accum, count, split_normals, cfg, out_arrays, out_capacity, n_out,
                action, workspace, stream=None):
    _check("veg_densify",
           load().veg_densify(ctypes.byref(in_arrays), n, _ptr(accum), _ptr(count),
                              _ptr(split_normals), cfg, ctypes.byref(out_arrays), out_capacity,
                              _ptr(n_out), _ptr(action), _ptr(workspace),
                              workspace.numel() * workspace.element_size(), _stream(stream)))


def veg_train_step(args, view, k, adam_step, accumulate_stats, stream=None):
    _check("veg_train_step", load().veg_train_step(ctypes.byref(args), view, k, adam_step,
                                                   1 if accumulate_stats else 0,
                                                   _stream(stream)))


def veg_volume_prepare(volume, vol4, stream=None):
    _check("veg_volume_prepare",
           load().veg_volume_prepare(_ptr(volume), volume.shape[0], _ptr(vol4), _stream(stream)))


def veg_raymarch(cams, vol4, tf, step, out, material=None, bg=(0.0, 0.0, 0.0), stats=None,
                 stream=None):
    """material: (k_a, k_d, k_s, beta) or None (unshaded)."""
    bgc = (ctypes.c_float * 3)(*[float(b) for b in bg])
    mat = None if material is None else ctypes.byref(veg_material(*[float(m) for m in material]))
    _check("veg_raymarch",
           load().veg_raymarch(cams, len(cams), _ptr(vol4), vol4.shape[0], tf, float(step), mat,
                               ctypes.cast(bgc, ctypes.c_void_p), _ptr(out), _ptr(stats),
                               _stream(stream)))


def veg_raymarch_cells_count(resolution, cell) -> int:
    c = ctypes.c_int64(0)
    _check("veg_raymarch_cells_count",
           load().veg_raymarch_cells_count(int(resolution), int(cell), ctypes.byref(c)))
    return int(c.value)


def veg_raymarch_cells(vol4, tf, cell, mask, stream=None):
    """mask: device int32/uint32 tensor of veg_raymarch_cells_count entries."""
    _check("veg_raymarch_cells",
           load().veg_raymarch_cells(_ptr(vol4), vol4.shape[0], tf, int(cell), _ptr(mask),
                                     _stream(stream)))


def veg_raymarch_masked(cams, vol4, tf, step, out, cell_mask, cell, material=None,
                        bg=(0.0, 0.0, 0.0), stats=None, stream=None):
    bgc = (ctypes.c_float * 3)(*[float(b) for b in bg])
    mat = None if material is None else ctypes.byref(veg_material(*[float(m) for m in material]))
    _check("veg_raymarch_masked",
           load().veg_raymarch_masked(cams, len(cams), _ptr(vol4), vol4.shape[0], tf, float(step),
                                      mat, ctypes.cast(bgc, ctypes.c_void_p), _ptr(cell_mask),
                                      int(cell), _ptr(out), _ptr(stats), _stream(stream)))


def veg_project_bwd(cams, g, tiles_touched, grad2d, grad_mean_v, grad_logscale_w, grad_quat,
                    stream=None):
    _check("veg_project_bwd",
           load().veg_project_bwd(cams, len(cams), g, _ptr(tiles_touched), _ptr(grad2d),
                                  _ptr(grad_mean_v), _ptr(grad_logscale_w), _ptr(grad_quat),
                                  _stream(stream)))


def veg_project_bwd_range(cams, g, tiles_touched, grad2d, first, count, grad_mean_v,
                          grad_logscale_w, grad_quat, stream=None):
    _check("veg_project_bwd_range",
           load().veg_project_bwd_range(cams, len(cams), g, _ptr(tiles_touched), _ptr(grad2d),
                                        int(first), int(count), _ptr(grad_mean_v),
                                        _ptr(grad_logscale_w), _ptr(grad_quat), _stream(stream)))


def veg_l1_loss_workspace_size() -> int:
    out = _SZ()
    _check("veg_l1_loss_workspace_size", load().veg_l1_loss_workspace_size(ctypes.byref(out)))
    return out.value


def veg_l1_loss(out, target, n_records, grad, loss, workspace, stream=None):
    _check("veg_l1_loss",
           load().veg_l1_loss(_ptr(out), _ptr(target), n_records, _ptr(grad), _ptr(loss),
                              _ptr(workspace), workspace.numel() * workspace.element_size(),
                              _stream(stream)))


def veg_render_workspace_size(n, n_views, capacity, width, height) -> int:
    out = _SZ()
    _check("veg_render_workspace_size",
           load().veg_render_workspace_size(n, n_views, capacity, width, height,
                                            ctypes.byref(out)))
    return out.value


def veg_render(cams, g, tf, bg, capacity, workspace, out, n_contrib, stream=None, tf_group=0):
    bgc = (ctypes.c_float * 3)(*[float(b) for b in bg])
    _check("veg_render",
           load().veg_render(cams, len(cams), g, tf, ctypes.cast(bgc, ctypes.c_void_p), tf_group,
                             capacity, _ptr(workspace), workspace.numel(), _ptr(out),
                             _ptr(n_contrib), _stream(stream)))
