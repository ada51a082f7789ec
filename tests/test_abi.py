"""The C ABI library builds, loads and exports every symbol declared in
include/veg.h; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re
import shutil

import pytest

from paper_2504_13339_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "veg.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(veg_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2504_13339_gb300 import build
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("veg_project", "veg_bin_sort", "veg_composite_fwd", "veg_composite_bwd",
                 "veg_render", "veg_sync_status", "veg_status_string", "veg_l1_loss",
                 "veg_shade", "veg_shade_bwd"):
        assert name in syms


def test_every_declared_symbol_is_exported_and_bound(lib):
    raw = ctypes.CDLL(_lib.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(raw, name), name
        assert name in _lib.EXPORTED, f"{name} has no binding"


def test_status_strings(lib):
    assert _lib.veg_status_string(0) == "ok"
    assert "capacity" in _lib.veg_status_string(2)
    assert _lib.veg_status_string(99) == "unknown status"
    assert isinstance(_lib.veg_kernel_launches(), int)


def test_host_side_validation_needs_no_gpu(lib):
    out = ctypes.c_size_t()
    assert lib.veg_bin_sort_workspace_size(-1, 1, 10, 64, 64, ctypes.byref(out)) == 1
    assert lib.veg_bin_sort_workspace_size(10, 0, 10, 64, 64, ctypes.byref(out)) == 1
    assert lib.veg_bin_sort_workspace_size(10, 1, 1 << 31, 64, 64, ctypes.byref(out)) == 1
    assert lib.veg_bin_sort_workspace_size(10, 1, 10, 0, 64, ctypes.byref(out)) == 1
    assert lib.veg_bin_sort_workspace_size(10, 1, 100, 64, 64, ctypes.byref(out)) == 0
    assert out.value > 0
    assert lib.veg_render_workspace_size(100, 2, 1000, 100, 70, ctypes.byref(out)) == 0
    assert lib.veg_composite_bwd_workspace_size(100, 2, ctypes.byref(out)) == 0
    assert out.value >= 2 * 100 * 2 * 16
    g = _lib.veg_gaussians(0, 0, 0, 10)
    # no cameras / zero views / bad image size: rejected before any launch
    assert lib.veg_project(None, 1, g, None, None, None, None, None, None) == 1
    cams = (_lib.veg_camera * 1)()
    cams[0].width, cams[0].height, cams[0].fx, cams[0].fy = 0, 64, 10.0, 10.0
    assert lib.veg_project(cams, 1, g, None, None, None, None, None, None) == 1
    cams[0].width = 64
    assert lib.veg_project(cams, 0, g, None, None, None, None, None, None) == 1
    # null Gaussian arrays with n > 0
    assert lib.veg_project(cams, 1, g, None, None, None, None, None, None) == 1
    tf = _lib.veg_tf(0, 1, 1)
    assert lib.veg_composite_fwd(cams, 1, 0, None, None, None, None, None, None, tf, None, 0, 0,
                                 None, None, None, None) == 1
    assert lib.veg_tile_order(None, 5, None, None) == 1
    assert lib.veg_sync_status(None, None, None) == 1
    # the fixed-scratch binning refuses a request beyond its array on the host
    fake = 1 << 20  # aligned placeholder addresses, never dereferenced
    assert lib.veg_bin_sort_static(cams, 1, 4096, fake, fake, fake, 4_000_000, None, fake,
                                   fake, None, None) == 5
    assert lib.veg_bin_sort_static(cams, 1, -1, fake, fake, fake, 16, None, fake, fake, None,
                                   None) == 1
    assert lib.veg_l1_loss(None, None, 4, None, None, None, 0, None) == 1
    # the tile batch is 0 (default), 128, 256 or 512
    tf1 = _lib.veg_tf(fake, 16, 1)
    assert lib.veg_composite_fwd(cams, 1, 0, None, None, None, None, fake, None, tf1, None, 0,
                                 100, fake, fake, None, None) == 1
    # shading: light directions are checked on the host; n = 0 launches nothing
    light = (ctypes.c_float * 3)(0.0, 0.0, 1.0)
    zero = (ctypes.c_float * 3)(0.0, 0.0, 0.0)
    assert lib.veg_shade(cams, 1, fake, 8, fake, fake, zero, fake, None) == 1
    assert lib.veg_shade(cams, 1, fake, 8, fake, fake, None, fake, None) == 1
    assert lib.veg_shade(cams, 1, fake, -1, fake, fake, light, fake, None) == 1
    assert lib.veg_shade(cams, 1, fake + 4, 8, fake, fake, light, fake, None) == 1
    assert lib.veg_shade(cams, 1, None, 0, None, None, light, None, None) == 0
    assert lib.veg_shade_bwd(cams, 1, fake, 8, fake, fake, light, None, fake, fake, fake, fake,
                             None) == 1
    assert lib.veg_shade_bwd(cams, 1, fake, 8, fake, fake, light, fake, fake, fake + 8, fake,
                             fake, None) == 1
    # Adam: the device step counter must be given and 16-byte aligned
    arrays = _lib.veg_adam_arrays()
    lrs = (ctypes.c_float * 20)()
    assert lib.veg_adam_step_counted(ctypes.byref(arrays), 0, lrs, 0.9, 0.999, 1e-15, None,
                                     None) == 1
    assert lib.veg_adam_step_counted(ctypes.byref(arrays), 0, lrs, 0.9, 0.999, 1e-15, fake + 8,
                                     None) == 1
    assert lib.veg_adam_step(ctypes.byref(arrays), 0, lrs, 0.9, 0.999, 1e-15, 0, None) == 1
    # raymarching: the mask's cell size is checked on the host
    tf16 = _lib.veg_tf(fake, 16, 1)
    assert lib.veg_raymarch_cells(fake, 16, tf16, 3, fake, None) == 1
    assert lib.veg_raymarch_cells(fake, 16, tf16, 128, fake, None) == 1
    assert lib.veg_raymarch_masked(cams, 1, fake, 16, tf16, 0.1, None, None, fake, 3, fake,
                                   None, None) == 1
    # the raymarcher's views share one size; the splatting entry points take
    # views of different sizes
    cams2 = (_lib.veg_camera * 2)()
    for c, (w, h) in zip(cams2, ((64, 48), (32, 32))):
        c.width, c.height, c.fx, c.fy = w, h, 40.0, 40.0
    assert lib.veg_raymarch_masked(cams2, 2, fake, 16, tf16, 0.1, None, None, fake, 8, fake,
                                   None, None) == 1
    assert lib.veg_project(cams2, 2, _lib.veg_gaussians(0, 0, 0, 0), None, None, None, None,
                           None, None) == 0  # n = 0: nothing to launch
    # per-view models: the list must be given and each model fit the stride
    ms = (_lib.veg_gaussians * 2)(_lib.veg_gaussians(fake, fake, fake, 10),
                                  _lib.veg_gaussians(fake, fake, fake, 30))
    assert lib.veg_project_views(cams2, 2, None, 30, None, fake, fake, fake, fake, None) == 1
    assert lib.veg_project_views(cams2, 2, ms, 20, None, fake, fake, fake, fake, None) == 1
    ms[1] = _lib.veg_gaussians(0, 0, 0, 30)  # null arrays with n > 0
    assert lib.veg_project_views(cams2, 2, ms, 30, None, fake, fake, fake, fake, None) == 1
    ms[1] = _lib.veg_gaussians(fake + 4, fake, fake, 30)  # misaligned
    assert lib.veg_project_views(cams2, 2, ms, 30, None, fake, fake, fake, fake, None) == 1
    ms[0] = ms[1] = _lib.veg_gaussians(0, 0, 0, 0)
    assert lib.veg_project_views(cams2, 2, ms, 0, None, None, None, None, None, None) == 0
    # veg_render: the TF group is 0 (default) or 1..8
    assert lib.veg_render(cams, 1, g, tf16, None, 9, 16, fake, 1 << 30, fake, fake, None) == 1


def test_raymarch_cell_count_host_logic(lib):
    from paper_2504_13339_gb300 import _lib
    assert _lib.veg_raymarch_cells_count(256, 8) == 32 ** 3
    assert _lib.veg_raymarch_cells_count(19, 4) == 5 ** 3
    assert _lib.veg_raymarch_cells_count(2, 1) == 1
    for bad in ((256, 3), (256, 0), (256, 128), (1, 4), (4096, 8)):
        with pytest.raises(RuntimeError):
            _lib.veg_raymarch_cells_count(*bad)
