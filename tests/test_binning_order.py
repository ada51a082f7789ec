"""The two-stage binning order (no GPU).

The GPU path sorts the (view, Gaussian) records by float32 depth bits
(stable, so ties keep index order), emits each record's tiles in that order
and stable-sorts the instances by (view, tile) alone.  This gives the order
of one stable sort of the 64-bit keys (view, tile, depth bits) of instances
emitted in index order (Sec. 3.3: lists sorted by tile and depth).  Checked
here on random records with heavy depth ties, several views and empty
records.
"""
import numpy as np
import pytest


def one_stage(depth_bits, rects, n, tiles_x, tb):
    keys, vals = [], []
    for r in range(len(depth_bits)):
        x0, y0, x1, y1 = rects[r]
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                keys.append((int(r // n) << (tb + 32)) | ((ty * tiles_x + tx) << 32)
                            | int(depth_bits[r]))
                vals.append(r)
    keys = np.array(keys, np.uint64)
    o = np.argsort(keys, kind="stable")
    return keys[o], np.array(vals, np.int64)[o]


def two_stage(depth_bits, rects, n, tiles_x, tiles_per_view):
    order = np.argsort(depth_bits, kind="stable")
    tkeys, vals = [], []
    for r in order:
        x0, y0, x1, y1 = rects[r]
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                tkeys.append((r // n) * tiles_per_view + ty * tiles_x + tx)
                vals.append(r)
    tkeys = np.array(tkeys, np.int64)
    o = np.argsort(tkeys, kind="stable")
    return tkeys[o], np.array(vals, np.int64)[o]


@pytest.mark.parametrize("seed", range(8))
def test_two_stable_stages_give_the_64_bit_key_order(seed):
    rng = np.random.default_rng(seed)
    views, n = int(rng.integers(1, 4)), int(rng.integers(1, 300))
    tiles_x, tiles_y = int(rng.integers(1, 9)), int(rng.integers(1, 7))
    tpv = tiles_x * tiles_y
    tb = max(1, int(np.ceil(np.log2(max(tpv, 2)))))
    # few distinct depths: many ties that only the index order breaks
    depth = rng.choice(np.float32([0.5, 1.25, 2.0, 2.0000002, 3.75]), views * n)
    bits = depth.view(np.uint32).astype(np.int64)
    x0 = rng.integers(0, tiles_x, views * n)
    y0 = rng.integers(0, tiles_y, views * n)
    x1 = np.minimum(x0 + rng.integers(0, 3, views * n), tiles_x)  # some empty
    y1 = np.minimum(y0 + rng.integers(1, 3, views * n), tiles_y)
    rects = np.stack([x0, y0, x1, y1], 1)
    k64, v1 = one_stage(bits, rects, n, tiles_x, tb)
    tk, v2 = two_stage(bits, rects, n, tiles_x, tpv)
    assert np.array_equal(v1, v2)
    view = (k64 >> np.uint64(tb + 32)).astype(np.int64)
    tile = ((k64 >> np.uint64(32)) & np.uint64((1 << tb) - 1)).astype(np.int64)
    assert np.array_equal(view * tpv + tile, tk)
