"""Tile-batch autotuner for the compositing kernels.

The compositor processes a group of TFs per pass over each tile's list
(`tf_group` = 1, 2, 4 or 8 for the forward, up to 4 for the backward),
staging the list in batches of `tile_batch` splats (128, 256 or 512)
through shared memory.  A larger group shares each splat's geometry across
more TFs but holds more state per pixel (registers) and more tables in
shared memory; a larger batch takes fewer block barriers per list but more
shared memory, and so fewer resident CTAs.  The best pair depends on the
number of TFs, the image and the scene.  `tune` times every admissible
(group, batch) pair on the caller's actual buffers with CUDA events and
returns the fastest; results are cached per (device, problem signature) in
a JSON file so a shape is tuned once.
"""
from __future__ import annotations

import json
import os

import torch

FWD_GROUPS = (1, 2, 4, 8)
BWD_GROUPS = (1, 2, 4)
BATCHES = (128, 256, 512)


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


def _best(times, prefix):
    """The fastest (group, batch) among the keys '<prefix><group>x<batch>'."""
    t, key = min((t, k) for k, t in times.items() if k.startswith(prefix))
    g, b = key[len(prefix):].split("x")
    return int(g), int(b)


def tune(p, luts, dout=None, reps=3, use_cache=True):
    """Chooses p.tf_group and p.tile_batch (forward), p.tf_group_bwd and
    p.tile_batch_bwd (backward, with `dout`) for pipeline `p` whose binning
    is current (project + bin_sort already run).  Returns {"fwd": group,
    "fwd_batch": batch, "bwd": group, "bwd_batch": batch, "times": ...}."""
    n_tf = luts.shape[0]
    key = signature(p, n_tf) + ("|bwd" if dout is not None else "") + "|batch"
    cache = _load() if use_cache else {}
    if key in cache:
        res = cache[key]
    else:
        times = {}
        for g in FWD_GROUPS:
            if g > 1 and g // 2 >= n_tf:
                continue
            for b in BATCHES:
                p.tf_group, p.tile_batch = g, b
                times[f"fwd{g}x{b}"] = _time(lambda: p.composite(luts), reps)
        fwd, fwd_b = _best(times, "fwd")
        p.tf_group, p.tile_batch = fwd, fwd_b
        p.composite(luts)
        bwd, bwd_b = 4, 256
        if dout is not None:
            for g in BWD_GROUPS:
                if g > 1 and g // 2 >= n_tf:
                    continue
                for b in BATCHES:
                    p.tf_group_bwd, p.tile_batch_bwd = g, b
                    times[f"bwd{g}x{b}"] = _time(lambda: p.backward_2d(dout), reps)
            bwd, bwd_b = _best(times, "bwd")
        res = {"fwd": fwd, "fwd_batch": fwd_b, "bwd": bwd, "bwd_batch": bwd_b, "times": times}
        if use_cache:
            cache[key] = res
            _store(cache)
    p.tf_group, p.tile_batch = res["fwd"], res["fwd_batch"]
    p.tf_group_bwd, p.tile_batch_bwd = res["bwd"], res["bwd_batch"]
    return res
