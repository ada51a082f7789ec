"""Pins of the oracle's threshold windows (reading R12) and of the outcome
explorer that checks flagged pixels (pixel_alternatives).

Eq. 1 with the skip, clamp and stop rules of Sec. 3.3 has four decisions
whose float32 and float64 evaluations can differ when they sit on a
threshold: the sign of the exponent, alpha >= 1/255, alpha = min(0.99, .)
and T (1 - alpha) >= 1e-4.  Each pin builds a splat (or two) whose decision
lies just inside or just outside its window and checks the flag, and that
the explorer lists both sides of an inside decision with the closed-form
outcome of each side.  Windows: relative 1e-5 for the two alpha tests,
relative 1e-3 for the stop, |exponent| <= 1e-5 of its terms."""
import math

import numpy as np
import pytest

from oracle import veg_oracle as O
from paper_2504_13339_gb300 import scenes as S

BG = np.array([0.2, 0.3, 0.4])
RGB = np.array([0.9, 0.4, 0.1])
RGB32 = RGB.astype(np.float32).astype(np.float64)  # the table's entries


def _two_entry_tf(a0, a1, rgb=RGB):
    """Table of two entries: v = 0 -> opacity a0, v = 1 -> opacity a1."""
    return np.array([[*rgb, a0], [*rgb, a1]], np.float32)[None].astype(np.float64)


def _run(u, conic, v, w, tf, px=8.0, py=8.0):
    u = np.asarray(u, np.float64).reshape(-1, 2)
    conic = np.asarray(conic, np.float64).reshape(-1, 3)
    v = np.asarray(v, np.float64).reshape(-1)
    w = np.asarray(w, np.float64).reshape(-1)
    r = O.composite_tile(np.array([px]), np.array([py]), u, conic, v, w, tf, BG)
    alts = O.pixel_alternatives(px, py, u, conic, v, w, tf[0], BG)
    return r, alts


def _single(opacity):
    """One splat centred on the pixel (exponent exactly 0, G = 1): alpha is
    the table's opacity itself."""
    tf = _two_entry_tf(opacity, opacity)
    return _run([8.0, 8.0], [1.0, 0.0, 1.0], [0.5], [1.0], tf)


# ----------------------------------------------------------------------------
# alpha = 1/255 (skip)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("rel,flagged", [(5e-6, True), (-5e-6, True), (2e-5, False),
                                         (-2e-5, False)])
def test_alpha_min_window(rel, flagged):
    a = (1.0 / 255.0) * (1.0 + rel)
    r, alts = _single(a)
    assert bool(r["flag"][0, 0]) == flagged
    a32 = float(np.float32(a))
    blended = np.concatenate([a32 * RGB32 + (1 - a32) * BG, [1 - a32]])
    skipped = np.concatenate([BG, [1.0]])
    by_n = {x["n_contrib"]: x["out"] for x in alts}
    if flagged:  # both sides, each in closed form
        assert len(alts) == 2 and sorted(by_n) == [0, 1]
        np.testing.assert_allclose(by_n[0], skipped, rtol=1e-12)
        np.testing.assert_allclose(by_n[1], blended, rtol=1e-12)
    else:  # one outcome, the float64 decision of composite_tile
        assert len(alts) == 1
        np.testing.assert_allclose(alts[0]["out"], r["out"][0, 0], rtol=1e-12)
        assert alts[0]["n_contrib"] == r["n_contrib"][0, 0] == (1 if rel > 0 else 0)


# ----------------------------------------------------------------------------
# alpha = 0.99 (clamp): alpha is 0.99 to within 1e-5 either way, so the
# outcome is not branched; the pixel is flagged and the outcome marked
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("rel,flagged", [(5e-6, True), (-5e-6, True), (2e-5, False),
                                         (-2e-5, False)])
def test_alpha_clamp_window(rel, flagged):
    r, alts = _single(0.99 * (1.0 + rel))
    assert bool(r["flag"][0, 0]) == flagged
    assert len(alts) == 1 and alts[0]["clamp_near"] == flagged
    assert alts[0]["clamped"][0] == (rel > 0)
    np.testing.assert_allclose(alts[0]["out"], r["out"][0, 0], rtol=1e-12)


# ----------------------------------------------------------------------------
# T (1 - alpha) = 1e-4 (stop): splats of alpha 0.95 and 0.85 leave T = 0.0075,
# then one of alpha = 1 - (1e-4 / 0.0075)(1 + rel) ~ 0.987 (below the clamp),
# so that T (1 - alpha) = 1e-4 (1 + rel)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("rel,flagged", [(5e-4, True), (-5e-4, True), (2e-3, False),
                                         (-2e-3, False)])
def test_transmittance_stop_window(rel, flagged):
    a1, a2 = float(np.float32(0.95)), float(np.float32(0.85))
    T2 = (1 - a1) * (1 - a2)
    a3 = float(np.float32(1.0 - 1e-4 * (1.0 + rel) / T2))
    tf = np.array([[*RGB, a3], [*RGB, a2], [*RGB, a1]], np.float32)[None].astype(np.float64)
    r, alts = _run([[8.0, 8.0]] * 3, [[1.0, 0.0, 1.0]] * 3, [1.0, 0.5, 0.0], [1.0] * 3, tf)
    assert bool(r["flag"][0, 0]) == flagged
    c2 = a1 + (1 - a1) * a2
    stop = np.concatenate([c2 * RGB32 + T2 * BG, [T2]])
    go = np.concatenate([(c2 + T2 * a3) * RGB32 + T2 * (1 - a3) * BG, [T2 * (1 - a3)]])
    by_n = {x["n_contrib"]: x["out"] for x in alts}
    if flagged:
        assert sorted(by_n) == [2, 3]
        np.testing.assert_allclose(by_n[2], stop, rtol=1e-12)
        np.testing.assert_allclose(by_n[3], go, rtol=1e-12)
    else:
        assert len(alts) == 1
        n = 3 if rel > 0 else 2
        assert alts[0]["n_contrib"] == r["n_contrib"][0, 0] == n
        np.testing.assert_allclose(alts[0]["out"], go if n == 3 else stop, rtol=1e-12)
    assert all(x["out"][3] >= O.T_MIN for x in alts if x["n_contrib"] == 2)


# ----------------------------------------------------------------------------
# exponent = 0 (sign): the indefinite form (a, b, c) = (0.5, 0, -0.5) gives
# power = (dy^2 - dx^2) / 4 with terms of size ~4 at dx = 2, so the window
# is |power| <= 4e-5
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("power,flagged", [(1e-7, True), (-1e-7, True), (1e-4, False),
                                           (-1e-4, False)])
def test_exponent_sign_window(power, flagged):
    dx = 2.0
    dy = math.sqrt(dx * dx + 4.0 * power)
    tf = _two_entry_tf(0.5, 0.5)
    r, alts = _run([8.0 + dx, 8.0 + dy], [0.5, 0.0, -0.5], [0.5], [1.0], tf)
    assert bool(r["flag"][0, 0]) == flagged
    ns = sorted(x["n_contrib"] for x in alts)
    if flagged:
        assert ns == [0, 1]
        blended = [x for x in alts if x["n_contrib"] == 1][0]["out"]
        a = 0.5 * math.exp(power)
        np.testing.assert_allclose(blended, np.concatenate([a * RGB32 + (1 - a) * BG, [1 - a]]),
                                   rtol=1e-12)
    else:
        assert ns == [0 if power > 0 else 1]
        np.testing.assert_allclose(alts[0]["out"], r["out"][0, 0], rtol=1e-12)


# ----------------------------------------------------------------------------
# on a random scene: an unflagged pixel has exactly one outcome, the
# compositor's; a flagged pixel's outcomes include the compositor's
# ----------------------------------------------------------------------------

def test_alternatives_agree_with_the_compositor_on_a_scene():
    g = S.uniform_gaussians(700, 61, logscale_mean=-2.6)
    cams = [S.orbit_camera(20.0, 10.0, 3.0, 48, 40)]
    tfs = S.bump_tfs(2, 62)
    proj, bins, fwd = O.render(cams, g, tfs, bg=tuple(BG), record=True)
    cam = cams[0]
    luts = np.asarray(tfs, np.float64)
    rng = np.random.default_rng(63)
    checked = 0
    for t in range(2):
        for y, x in zip(rng.integers(0, cam.height, 60), rng.integers(0, cam.width, 60)):
            tile = (y // 16) * cam.tiles_x + x // 16
            lo, hi = bins["ranges"][0, tile]
            idx, u, conic, v, w = O._tile_splats(proj[0], bins["vals"], lo, hi, g.n)
            alts = O.pixel_alternatives(x, y, u, conic, v, w, luts[t], BG)
            ref = fwd["out"][0, t, y, x]
            match = [a for a in alts if a["n_contrib"] == fwd["n_contrib"][0, t, y, x]
                     and np.allclose(a["out"], ref, rtol=1e-12, atol=1e-15)]
            assert match, (t, y, x)
            if not fwd["flag"][0, t, y, x]:
                assert len(alts) == 1
            # the recorded decisions are the matching outcome's
            p = O.tile_pixel_index(cam, tile, x, y)
            rec = fwd["rec"][0, tile]
            blend = np.array([rec[i][0][p, t] for i in range(len(rec))], bool)
            assert any(np.array_equal(a["blend"][:len(rec)], blend) and
                       not a["blend"][len(rec):].any() for a in match)
            checked += 1
    assert checked == 120


def test_flag_alternatives_cover_every_flagged_pixel():
    g = S.uniform_gaussians(900, 64, logscale_mean=-2.4)
    cams = [S.orbit_camera(35.0, -15.0, 3.0, 64, 48)]
    tfs = S.bump_tfs(3, 65)
    proj, bins, fwd = O.render(cams, g, tfs, record=True)
    alts = O.flag_alternatives(proj, cams, bins, tfs, (0.0, 0.0, 0.0), fwd)
    assert len(alts) == int(fwd["flag"].sum())
    for (vi, t, y, x), a in alts.items():
        assert a is not None
        ref = fwd["out"][vi, t, y, x]
        assert any(np.allclose(o["out"], ref, rtol=1e-12, atol=1e-15) and
                   o["n_contrib"] == fwd["n_contrib"][vi, t, y, x] for o in a)
