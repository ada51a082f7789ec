"""The parity helpers of the GPU tests (tests/parity.py), checked on the CPU
with simulated kernel outputs: a kernel that took the other side of every
flagged decision is accepted and the oracle's recorded decisions follow it;
a pixel off by more than the bar is not; the element-wise gradient bound
catches an error on a small entry that the per-tensor bound lets through."""
import numpy as np
import pytest

from oracle import veg_oracle as O
from paper_2504_13339_gb300 import scenes as S
import parity


def _scene():
    g = S.uniform_gaussians(1500, 70, logscale_mean=-2.5)
    cams = [S.orbit_camera(20.0, 10.0, 3.0, 64, 48)]
    tfs = S.bump_tfs(3, 71)
    proj, bins, fwd = O.render(cams, g, tfs, record=True)
    return g, cams, tfs, proj, bins, fwd


def _other_side(proj, cams, bins, tfs, fwd):
    """A simulated kernel output: float32 images that took, at every flagged
    pixel, an outcome other than the float64 one."""
    out = fwd["out"].astype(np.float32)
    nc = fwd["n_contrib"].astype(np.int32)
    taken = {}
    for key, alts in O.flag_alternatives(proj, cams, bins, tfs, (0, 0, 0), fwd).items():
        ref = fwd["out"][key]
        other = [a for a in alts if not (a["n_contrib"] == fwd["n_contrib"][key]
                                         and np.allclose(a["out"], ref, rtol=0, atol=1e-12))]
        if other:
            out[key] = other[0]["out"]
            nc[key] = other[0]["n_contrib"]
            taken[key] = other[0]
    return out, nc, taken


def test_flagged_pixels_follow_the_kernels_decisions():
    g, cams, tfs, proj, bins, fwd = _scene()
    cam = cams[0]
    out, nc, taken = _other_side(proj, cams, bins, tfs, fwd)
    assert len(taken) >= 20
    # a splat that a resolved pixel blends where the float64 decisions skip
    # it (or the reverse), read from the recorded decisions before resolving
    flips = []
    for (vi, t, y, x), alt in taken.items():
        tile = (y // 16) * cam.tiles_x + x // 16
        p = O.tile_pixel_index(cam, tile, x, y)
        rec = fwd["rec"][vi, tile]
        before = np.array([r[0][p, t] for r in rec], bool)
        for k in np.nonzero(before != alt["blend"][:len(rec)])[0]:
            lo = bins["ranges"][vi, tile][0]
            flips.append(int(bins["vals"][lo + k]) % g.n)
    assert flips
    excl = parity.checked_forward("cpu_simulated", fwd, proj, cams, bins, tfs, (0, 0, 0), out,
                                  nc)
    for (vi, t, y, x), alt in taken.items():
        assert fwd["n_contrib"][vi, t, y, x] == alt["n_contrib"]
        np.testing.assert_allclose(fwd["out"][vi, t, y, x], alt["out"], rtol=0, atol=0)
        tile = (y // 16) * cam.tiles_x + x // 16
        p = O.tile_pixel_index(cam, tile, x, y)
        rec = fwd["rec"][vi, tile]
        assert np.array_equal([r[0][p, t] for r in rec], alt["blend"][:len(rec)])
    assert excl.sum() <= 1
    # the backward over the rewritten decisions is the gradient of the render
    # with those decisions frozen: central differences in a flipped splat's
    # weight
    dout = np.random.default_rng(72).standard_normal(fwd["out"].shape)
    dout[excl] = 0.0
    g2 = O.composite_bwd(proj, cams, bins, tfs, (0, 0, 0), fwd, dout)
    mean = g.mean_v[:, :3].astype(np.float64)
    v = g.mean_v[:, 3].astype(np.float64)
    ls = g.logscale_w[:, :3].astype(np.float64)
    w = g.logscale_w[:, 3].astype(np.float64)
    q = g.quat.astype(np.float64)
    tiles = list(range(cam.tiles_x * cam.tiles_y))
    i = max(set(flips), key=lambda j: abs(g2[0, j, 6]))
    assert g2[0, i, 6] != 0.0
    h = 1e-6
    vals = []
    for sgn in (1.0, -1.0):
        wp = w.copy()
        wp[i] += sgn * h
        f = O.render_frozen(cams, mean, ls, q, v, wp, tfs, (0, 0, 0), bins, fwd["rec"], tiles)
        vals.append(float((f * dout).sum()))
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(fd - g2[0, i, 6]) <= 1e-6 * max(1.0, abs(fd))


def test_a_pixel_off_the_bar_is_not_accepted():
    g, cams, tfs, proj, bins, fwd = _scene()
    out = fwd["out"].astype(np.float32)
    nc = fwd["n_contrib"].astype(np.int32)
    key = tuple(int(k) for k in np.argwhere(fwd["flag"])[0])
    out[key][0] += 2.5e-4
    with pytest.raises(AssertionError):
        parity.resolve("cpu_planted", fwd, proj, cams, bins, tfs, (0, 0, 0), out, nc)
    parity.REPORT.pop()


def test_elementwise_gradient_bound():
    n0 = len(parity.GRAD_RATIOS)
    rng = np.random.default_rng(73)
    ref = rng.standard_normal(1000)
    ref[:10] *= 1e-5  # small entries
    got = ref * (1 + 1e-5)
    parity.grad_check(got, ref, "close")
    bad = got.copy()
    bad[3] = ref[3] + 5e-4 * np.abs(ref).max()  # within the per-tensor bar only
    assert np.abs(bad - ref).max() <= parity.GRAD_TOL * np.abs(ref).max()
    with pytest.raises(AssertionError):
        parity.grad_check(bad, ref, "planted")
    del parity.GRAD_RATIOS[n0:]  # keep the run's report to the real tensors
