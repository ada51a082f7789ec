"""VEG adaptive density control oracle: clone, split and prune (Sec. 4.2).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA library and never calls it.

What it computes.  The paper densifies and prunes "following the method of
Kerbl and Kopanas et al." (3D Gaussian splatting): a Gaussian whose averaged
view-space positional gradient is large sits in a poorly reconstructed region
and is cloned (small Gaussians) or split in two (large ones, children drawn
from the Gaussian itself as a density, scale divided by 1.6); Gaussians of low
weight w are removed (the paper's threshold 0.005 on w instead of opacity),
from iteration 500 to 20,000.

Readings where the paper is silent (listed in the design notes):
  R20 statistic: for every view in which a Gaussian touches a tile, the norm
      of its screen-mean gradient in normalised device units,
      |(dL/du_x W/2, dL/du_y H/2)|, is added to an accumulator and a count is
      incremented; the average accumulator / count is compared with 0.0002.
      Accumulation is float32 in view order; every product, sum, square root
      and quotient is rounded separately (no fused multiply-add), so decisions
      are reproducible bit for bit.
  R21 decisions (float32, thresholds rounded to float32 once):
      prune  if w_raw < logit(0.005)           (w = sigmoid(w_raw) < 0.005);
      else, if the average is >= 0.0002:
        split  if max(log-scale) > ln(0.01 extent)   (3DGS's percent-dense
               rule, extent = 1.1 x the largest distance of a training camera
               from the cameras' centroid),
        clone  otherwise;
      else keep.
  R22 outputs, in input order: keep -> the Gaussian; clone -> the Gaussian,
      then its copy; split -> two children, the parent removed; prune -> none.
      A split child j takes mu + R(q) diag(s) z_j (z_j given standard normal
      samples), log-scale - ln 1.6, and every other value of the parent.
      Adam moments: kept Gaussians and the first of a clone pair keep theirs,
      copies and children start at zero.  The statistics restart at zero.
"""
from __future__ import annotations

import math

import numpy as np

from .veg_oracle import _quat_rot64

F = np.float32

GRAD_THRESHOLD = 0.0002
DENSE_FRACTION = 0.01
PRUNE_WEIGHT = 0.005
SPLIT_FACTOR = 1.6
SPLIT_CHILDREN = 2

PRUNE, KEEP, CLONE, SPLIT = 0, 1, 2, 3


def grad_stat_update(accum, count, grad2d_uv, tiles, width, height):
    """Adds one iteration's views to the statistics (reading R20).

    accum (N,) float32, count (N,) int32 (updated in place); grad2d_uv
    (V, N, 2) float32 dL/du; tiles (V, N) tiles touched."""
    hx, hy = F(0.5 * width), F(0.5 * height)
    V, N = tiles.shape
    for v in range(V):
        vis = tiles[v] > 0
        gx = (grad2d_uv[v, :, 0].astype(F) * hx).astype(F)
        gy = (grad2d_uv[v, :, 1].astype(F) * hy).astype(F)
        nrm = np.sqrt((gx * gx).astype(F) + (gy * gy).astype(F)).astype(F)
        accum[vis] = (accum[vis] + nrm[vis]).astype(F)
        count[vis] += 1
    return accum, count


def scene_extent(cam_centres):
    c = np.asarray(cam_centres, np.float64)
    return 1.1 * float(np.linalg.norm(c - c.mean(0), axis=1).max())


def thresholds(extent, grad_threshold=GRAD_THRESHOLD, dense_fraction=DENSE_FRACTION,
               prune_weight=PRUNE_WEIGHT):
    """The float32 thresholds of reading R21."""
    return {"grad": F(grad_threshold),
            "log_size": F(math.log(dense_fraction * extent)),
            "raw_weight": F(math.log(prune_weight) - math.log1p(-prune_weight)),
            "log_split": F(math.log(SPLIT_FACTOR))}


def classify(raw_logscale_w, accum, count, th):
    """Action per Gaussian (PRUNE, KEEP, CLONE, SPLIT)."""
    lw = np.asarray(raw_logscale_w, F)
    avg = np.where(count > 0, (accum.astype(F) / np.maximum(count, 1).astype(F)).astype(F),
                   F(0.0))
    act = np.full(lw.shape[0], KEEP, np.int32)
    hot = avg >= th["grad"]
    big = np.max(lw[:, :3], axis=1) > th["log_size"]
    act[hot & ~big] = CLONE
    act[hot & big] = SPLIT
    act[lw[:, 3] < th["raw_weight"]] = PRUNE
    return act


def densify(params, exp_avg, exp_avg_sq, accum, count, z, th):
    """Applies one densification (readings R21, R22).

    params / exp_avg / exp_avg_sq: lists of five (N, 4) arrays (raw mean_v,
    raw logscale_w, quat, normal_beta, k_ads; None entries skipped);
    z: (N, 2, 3) standard normal samples for split children.  Returns
    (new params, new exp_avg, new exp_avg_sq, actions)."""
    act = classify(params[1], accum, count, th)
    n = act.shape[0]
    q = np.asarray(params[2], np.float64)
    _, R = _quat_rot64(q)
    s = np.exp(np.asarray(params[1], np.float64)[:, :3])
    out_p = [[] for _ in range(5)]
    out_m = [[] for _ in range(5)]
    out_v = [[] for _ in range(5)]
    for i in range(n):
        if act[i] == PRUNE:
            continue
        if act[i] in (KEEP, CLONE):
            reps = [(None, True)] + ([(None, False)] if act[i] == CLONE else [])
        else:
            reps = [(j, False) for j in range(SPLIT_CHILDREN)]
        for child, keep_state in reps:
            for a in range(5):
                if params[a] is None:
                    continue
                row = np.array(params[a][i], np.float64)
                if child is not None and a == 0:
                    row[:3] = row[:3] + R[i] @ (s[i] * z[i, child])
                if child is not None and a == 1:
                    row[:3] = (np.asarray(params[1][i, :3], F) - th["log_split"]).astype(F)
                out_p[a].append(row)
                out_m[a].append(np.array(exp_avg[a][i]) if keep_state else np.zeros(4))
                out_v[a].append(np.array(exp_avg_sq[a][i]) if keep_state else np.zeros(4))
    stack = lambda rows, a: (None if params[a] is None else
                             (np.array(rows, np.float64).reshape(-1, 4)))
    return ([stack(out_p[a], a) for a in range(5)], [stack(out_m[a], a) for a in range(5)],
            [stack(out_v[a], a) for a in range(5)], act)
