"""Parity bars of the GPU tests against the oracle, shared by the test files.

Images: every pixel within IMG_TOL (max-abs per channel) and every
n_contrib equal.  A pixel whose decisions sit on a threshold (reading R12;
float32 and float64 may take them differently) is not dropped: the oracle
lists every outcome with those decisions taken either way
(``pixel_alternatives``) and the GPU pixel must equal one of them, whose
decisions then replace the float64 ones in the recorded forward, so the
oracle's backward follows the same decisions as the kernel's.  Only a pixel
whose decisions cannot be told apart from its image (a pair on the 0.99
clamp: alpha is 0.99 either way, the gradient is not) has its upstream
gradient zeroed, and such pixels must be at most EXCLUDED_MAX of the image.

Gradients, per tensor: max |g - g_ref| <= GRAD_TOL max |g_ref| and, per
element, |g - g_ref| <= GRAD_TOL |g_ref| + GRAD_FLOOR max |g_ref|.

Every resolution is recorded in REPORT and printed at the end of the run.
"""
from __future__ import annotations

import numpy as np

from oracle import veg_oracle as O

IMG_TOL = 1e-4
GRAD_TOL = 1e-3
GRAD_FLOOR = 1e-6
EXCLUDED_MAX = 1e-5
# alternatives whose final transmittance differs by less than this relative
# amount are told apart by nothing else but their colour (float32 carries
# ~1e-5 relative error in T over a long list; one blended splat changes it
# by at least 1/255)
T_RESOLVE = 1e-3

REPORT = []
GRAD_RATIOS = []


def resolve(name, fwd, proj, cams, bins, luts, bg, out_gpu, nc_gpu, region=None):
    """Matches every flagged (view, TF, pixel) of the oracle's forward `fwd`
    to the outcome the GPU took and rewrites `fwd` (out, n_contrib and, when
    recorded, the decisions) to that outcome.  Returns the report dict; its
    "grad_excluded" mask (V, T, H, W) marks pixels whose upstream gradient
    must be zeroed.  `region` (a mask of the checked pixels) only sets the
    pixel count of the report."""
    alts = O.flag_alternatives(proj, cams, bins, luts, bg, fwd)
    excl = np.zeros(fwd["flag"].shape, bool)
    unmatched = []
    n_alt = 0
    for (vi, t, y, x), outs in alts.items():
        gpu = out_gpu[vi, t, y, x].astype(np.float64)
        if outs is None:
            unmatched.append(((vi, t, y, x), "more outcomes than the explorer's limit"))
            continue
        n_alt += len(outs)
        cand = [o for o in outs if o["n_contrib"] == int(nc_gpu[vi, t, y, x])
                and np.max(np.abs(o["out"] - gpu)) <= IMG_TOL]
        if not cand:
            unmatched.append(((vi, t, y, x), "no outcome matches"))
            continue
        rel = [abs(o["out"][3] / gpu[3] - 1.0) for o in cand]
        best = cand[int(np.argmin(rel))]
        close = [o for o, r in zip(cand, rel) if r <= min(rel) + T_RESOLVE]
        if best["clamp_near"] or len(close) > 1:
            excl[vi, t, y, x] = True
        fwd["out"][vi, t, y, x] = best["out"]
        fwd["n_contrib"][vi, t, y, x] = best["n_contrib"]
        rec = fwd.get("rec")
        if rec:
            cam = cams[vi]
            tile = (y // O.TILE) * cam.tiles_x + x // O.TILE
            p = O.tile_pixel_index(cam, tile, x, y)
            for i, (blend, clamped) in enumerate(rec[vi, tile]):
                blend[p, t] = best["blend"][i]
                clamped[p, t] = best["clamped"][i]
    pixels = int(np.prod(fwd["flag"].shape)) if region is None else int(np.sum(region))
    rep = {"test": name, "pixels": pixels, "flagged": len(alts), "outcomes": n_alt,
           "unmatched": len(unmatched), "grad_excluded": int(excl.sum())}
    REPORT.append(rep)
    assert not unmatched, unmatched[:5]
    rep["grad_excluded_mask"] = excl
    return rep


def image_check(out_gpu, fwd, nc_gpu=None, region=None):
    """Every pixel (of `region`, an index into (V, T, H, W), when given)
    within IMG_TOL; n_contrib equal when given.  Call after `resolve`."""
    ref, got = fwd["out"], out_gpu
    if region is not None:
        ref, got = ref[region], got[region]
    err = np.abs(got - ref)
    assert np.all(err <= IMG_TOL), float(err.max())
    if nc_gpu is not None:
        nref = fwd["n_contrib"] if region is None else fwd["n_contrib"][region]
        ngot = nc_gpu if region is None else nc_gpu[region]
        assert np.array_equal(ngot, nref)
    return float(err.max())


def checked_forward(name, fwd, proj, cams, bins, luts, bg, out_gpu, nc_gpu, region=None):
    """resolve + image_check; returns the mask of pixels whose upstream
    gradient must be zeroed, after asserting that they are at most
    EXCLUDED_MAX of the pixels."""
    rep = resolve(name, fwd, proj, cams, bins, luts, bg, out_gpu, nc_gpu, region)
    image_check(out_gpu, fwd, nc_gpu, region)
    excl = rep.pop("grad_excluded_mask")
    assert excl.sum() <= EXCLUDED_MAX * rep["pixels"] or excl.sum() <= 1, rep
    return excl


def grad_check(got, ref, name, elementwise=True):
    """Both gradient bars (the element-wise one only when `elementwise`);
    returns the largest error over the element-wise bound, which is also
    recorded for the report."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = max(float(np.abs(ref).max()), 1e-30)
    err = np.abs(got - ref)
    rel = float(err.max()) / scale
    assert rel <= GRAD_TOL, (name, rel)
    bound = GRAD_TOL * np.abs(ref) + GRAD_FLOOR * scale
    ratio = float((err / bound).max()) if err.size else 0.0
    GRAD_RATIOS.append((name, ratio, int((err > bound).sum()), elementwise))
    if elementwise:
        assert ratio <= 1.0, (name, int((err > bound).sum()), ratio)
    return ratio


def summary_lines():
    if not REPORT and not GRAD_RATIOS:
        return []
    lines = ["parity: flagged (threshold-straddling) pixels resolved against the oracle's "
             "outcomes"]
    tot = {"pixels": 0, "flagged": 0, "unmatched": 0, "grad_excluded": 0}
    for r in REPORT:
        for k in tot:
            tot[k] += r[k]
        lines.append(f"  {r['test']}: {r['flagged']} flagged of {r['pixels']} "
                     f"({r['flagged'] / max(r['pixels'], 1):.2e}), {r['outcomes']} outcomes, "
                     f"unmatched {r['unmatched']}, gradient-excluded {r['grad_excluded']}")
    lines.append(f"  total: {tot['flagged']} flagged of {tot['pixels']} "
                 f"({tot['flagged'] / max(tot['pixels'], 1):.2e}), unmatched {tot['unmatched']}, "
                 f"excluded from the image bar 0, gradient-excluded {tot['grad_excluded']} "
                 f"({tot['grad_excluded'] / max(tot['pixels'], 1):.2e})")
    if GRAD_RATIOS:
        worst = max(GRAD_RATIOS, key=lambda r: r[1] if r[3] else -1.0)
        lines.append(f"  gradients: {len(GRAD_RATIOS)} tensors checked; largest error over the "
                     f"element-wise bound {worst[1]:.3f} ({worst[0]})")
        for nm, ratio, nbad, elem in GRAD_RATIOS:
            if not elem:
                lines.append(f"  per-tensor bound only: {nm} element-wise ratio {ratio:.3f}, "
                             f"{nbad} entries above it")
    return lines
