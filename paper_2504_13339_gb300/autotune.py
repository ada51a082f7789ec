"""Tile-batch autotuner for the compositing kernels.

The compositor processes a group of TFs per pass over each tile's list
(`tf_group` = 1, 2, 4 or 8 for the forward, up to 4 for the backward).  A
larger group shares each splat's geometry across more TFs but holds more
state per pixel (registers) and more tables in shared memory, so the best
size depends on the number of TFs, the image and the scene.  `tune` times
every admissible size on the caller's actual buffers with CUDA events and
returns the fastest; results are cached per (device, problem signature) in
a JSON file so a shape is tuned once.
"""
from __future__ import annotations

import json
import os

import torch

FWD_GROUPS = (1, 2, 4, 8)
BWD_GROUPS = (1, 2, 4)


def _cache_path():
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "veg_gb300", "autotune.json")


def _load():
    try:
        with open(_cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(cache):
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path + ".tmp", "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(path + ".tmp", path)
    except OSError:
        pass


def _time(fn, reps):
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    b.synchronize()
    return a.elapsed_time(b) / reps


def signature(p, n_tf):
    dev = torch.cuda.get_device_name(p.device)
    return f"{dev}|n={p.n}|V={p.V}|{p.W}x{p.H}|T={n_tf}|cap={p.capacity // (1 << 20)}"


def tune(p, luts, dout=None, reps=3, use_cache=True):
    """Chooses p.tf_group (forward) and p.tf_group_bwd for pipeline `p`
    whose binning is current (project + bin_sort already run).  With `dout`
    the backward is tuned too.  Returns {"fwd": g, "bwd": g, "times": ...}."""
    n_tf = luts.shape[0]
    key = signature(p, n_tf) + ("|bwd" if dout is not None else "")
    cache = _load() if use_cache else {}
    if key in cache:
        res = cache[key]
    else:
        times = {}
        for g in FWD_GROUPS:
            if g > 1 and g // 2 >= n_tf:
                continue
            p.tf_group = g
            times[f"fwd{g}"] = _time(lambda: p.composite(luts), reps)
        fwd = min((t, int(k[3:])) for k, t in times.items() if k.startswith("fwd"))[1]
        p.tf_group = fwd
        p.composite(luts)
        bwd = 4
        if dout is not None:
            for g in BWD_GROUPS:
                if g > 1 and g // 2 >= n_tf:
                    continue
                p.tf_group_bwd = g
                times[f"bwd{g}"] = _time(lambda: p.backward_2d(dout), reps)
            bwd = min((t, int(k[3:])) for k, t in times.items() if k.startswith("bwd"))[1]
        res = {"fwd": fwd, "bwd": bwd, "times": times}
        if use_cache:
            cache[key] = res
            _store(cache)
    p.tf_group = res["fwd"]
    p.tf_group_bwd = res["bwd"]
    return res
