"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms, a Monte-Carlo projection of sampled points, brute-force
enumeration, invariants and central finite differences."""
import json
import math
import os

import numpy as np
import pytest

from oracle import veg_oracle as O
from paper_2504_13339_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def make_gs(mean, logscale, quat=None, v=None, w=None):
    mean = np.atleast_2d(np.asarray(mean, np.float64))
    n = mean.shape[0]
    logscale = np.broadcast_to(np.asarray(logscale, np.float64), (n, 3))
    quat = np.tile([1.0, 0, 0, 0], (n, 1)) if quat is None else np.atleast_2d(quat)
    v = np.full(n, 0.5) if v is None else np.broadcast_to(np.asarray(v, np.float64), (n,))
    w = np.ones(n) if w is None else np.broadcast_to(np.asarray(w, np.float64), (n,))
    return S.Gaussians(np.concatenate([mean, v[:, None]], 1).astype(np.float32),
                       np.concatenate([logscale, w[:, None]], 1).astype(np.float32),
                       np.asarray(quat, np.float32))


# ----------------------------------------------------------------------------
# float32 exp (Cody-Waite)
# ----------------------------------------------------------------------------

def test_exp32_within_two_ulp():
    x = np.concatenate([np.linspace(-20, 20, 200001), [-1e-8, 0.0, 1e-8, 1.0, -3.5, -6.2]])
    x = x.astype(np.float32)
    got = O.exp32(x).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(got - ref) / ulp) <= 2.0
    assert O.exp32(np.float32(0.0)) == np.float32(1.0)


# ----------------------------------------------------------------------------
# transfer function (Sec. 3.3: linear interpolation between control points)
# ----------------------------------------------------------------------------

def test_tf_lerp_knots_segments_and_slope():
    rng = np.random.default_rng(0)
    L = 9
    lut = rng.uniform(0, 1, (L, 4)).astype(np.float32)
    knots = np.arange(L) / (L - 1)
    val, _ = O.tf_eval64(lut, knots)
    np.testing.assert_allclose(val, lut, atol=1e-15)
    v = rng.uniform(0, 1, 1000)
    val, slope = O.tf_eval64(lut, v)
    for c in range(4):  # equals numpy's piecewise-linear interpolation
        np.testing.assert_allclose(val[:, c], np.interp(v, knots, lut[:, c]), atol=1e-12)
    h = 1e-7
    fd = (O.tf_eval64(lut, v + h)[0] - O.tf_eval64(lut, v - h)[0]) / (2 * h)
    away = np.min(np.abs(v[:, None] - knots[None]), 1) > 1e-5
    np.testing.assert_allclose(slope[away], fd[away], rtol=1e-5, atol=1e-6)
    # outside [0,1] the value clamps and the slope is zero
    val, slope = O.tf_eval64(lut, np.array([-0.5, 1.5]))
    np.testing.assert_allclose(val, lut[[0, -1]], atol=1e-15)
    assert np.all(slope == 0)
    # float32 path agrees with float64 to float32 rounding
    v32 = rng.uniform(0, 1, 1000).astype(np.float32)
    np.testing.assert_allclose(O.tf_eval32(lut, v32), O.tf_eval64(lut, v32)[0], atol=3e-7)


# ----------------------------------------------------------------------------
# projection (Sec. 3.3: Sigma = R S S^T R^T, EWA Sigma' = J W Sigma W^T J^T)
# ----------------------------------------------------------------------------

def _hamilton_rotate(q, p):
    """Rotate p by unit quaternion q with quaternion products q p q*."""
    def mul(a, b):
        w1, x1, y1, z1 = a
        w2, x2, y2, z2 = b
        return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                         w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                         w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                         w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])
    qc = q * np.array([1, -1, -1, -1])
    return mul(mul(q, np.concatenate([[0.0], p])), qc)[1:]


def test_rotation_matrix_is_quaternion_rotation():
    rng = np.random.default_rng(1)
    q = rng.standard_normal((50, 4))
    qn, R = O._quat_rot64(q)
    for i in range(50):
        assert abs(np.linalg.det(R[i]) - 1) < 1e-12
        np.testing.assert_allclose(R[i] @ R[i].T, np.eye(3), atol=1e-12)
        p = rng.standard_normal(3)
        np.testing.assert_allclose(R[i] @ p, _hamilton_rotate(qn[i], p), atol=1e-12)


@pytest.mark.parametrize("width", [32, 128])
def test_isotropic_on_axis_closed_form(width):
    cam = S.look_at_camera((0, 0, 3), width, width)
    sigma = 0.05
    rng = np.random.default_rng(2)
    g = make_gs(np.zeros((4, 3)), math.log(sigma), quat=rng.standard_normal((4, 4)))
    f = cam.fx
    k = (f * sigma / 3.0) ** 2 + 0.3
    r_exp = math.ceil(3 * math.sqrt(k + math.sqrt(0.1)))
    p32 = O.project32(cam, g)
    p64 = O.project64(cam, g.mean_v[:, :3].astype(float), g.logscale_w[:, :3].astype(float),
                      g.quat.astype(float))
    for p in (p32["geo"][:, :2], p64["u"]):
        np.testing.assert_allclose(p, np.tile([cam.cx, cam.cy], (4, 1)), atol=1e-4)
    np.testing.assert_allclose(p32["geo"][:, 2], 3.0, rtol=1e-6)
    for con in (p32["aux"][:, :3], p64["conic"]):  # isotropic: independent of rotation
        np.testing.assert_allclose(con, np.tile([1 / k, 0.0, 1 / k], (4, 1)), rtol=1e-5,
                                   atol=1e-7)
    assert np.all(p32["radius"] == r_exp)


def test_off_axis_hand_derived_jacobian():
    cam = S.look_at_camera((0, 0, 3), 128, 128)
    f = cam.fx
    sigma = 0.03
    pts = np.array([[0.3, 0.2, 0.0], [-0.5, 0.4, 0.5], [0.1, -0.6, -0.4]])
    g = make_gs(pts, math.log(sigma))
    p64 = O.project64(cam, pts, np.full((3, 3), math.log(sigma)), np.tile([1.0, 0, 0, 0], (3, 1)))
    p32 = O.project32(cam, g)
    for i, (x, y, z) in enumerate(pts):
        X, Y, Z = x, -y, 3.0 - z  # camera frame of the look-at camera: (right, down, forward)
        JJ = np.array([[f * f / Z ** 2 + f * f * X * X / Z ** 4, f * f * X * Y / Z ** 4],
                       [f * f * X * Y / Z ** 4, f * f / Z ** 2 + f * f * Y * Y / Z ** 4]])
        Sp = sigma ** 2 * JJ + 0.3 * np.eye(2)
        Q = np.linalg.inv(Sp)
        ref = np.array([Q[0, 0], Q[0, 1], Q[1, 1]])
        np.testing.assert_allclose(p64["conic"][i], ref, rtol=1e-10)
        np.testing.assert_allclose(p32["aux"][i, :3], ref, rtol=2e-5, atol=1e-7)
        np.testing.assert_allclose(p64["u"][i], [f * X / Z + cam.cx, f * Y / Z + cam.cy],
                                   rtol=1e-12)


def test_jacobian_clamped_beyond_the_frustum():
    """Reading R2: x/z in the Jacobian is clamped to 1.3 tan(fov/2).  A
    large isotropic Gaussian centred right of the image (x/z = 1.2 times the
    limit) still reaches it; its conic is the closed form with the clamped
    x/z, about 5% away from the unclamped one."""
    cam = S.look_at_camera((0, 0, 3), 64, 64)
    f, Z = cam.fx, 3.0
    lim = 1.3 * 32.0 / f
    X = 1.2 * lim * Z
    sigma = 0.4
    ref = []
    for xc in (lim, X / Z):
        a = sigma ** 2 * f * f / Z ** 2 * (1.0 + xc * xc) + 0.3
        c = sigma ** 2 * f * f / Z ** 2 + 0.3
        ref.append(np.array([1.0 / a, 0.0, 1.0 / c]))
    assert abs(ref[0][0] / ref[1][0] - 1.0) > 0.03
    g = make_gs([[X, 0.0, 0.0]], math.log(sigma))
    p32 = O.project32(cam, g)
    p64 = O.project64(cam, np.array([[X, 0.0, 0.0]]), np.full((1, 3), math.log(sigma)),
                      np.array([[1.0, 0, 0, 0]]))
    assert p32["count"][0] > 0 and p32["geo"][0, 0] > cam.width  # centre off the image
    np.testing.assert_allclose(p32["aux"][0, :3], ref[0], rtol=2e-5, atol=1e-9)
    np.testing.assert_allclose(p64["conic"][0], ref[0], rtol=1e-10, atol=1e-14)


def test_tf_cull_threshold():
    """Reading R5: with the table given, a Gaussian is culled iff A(v) w <
    1/255 (here A = 0.5 everywhere); without it nothing is culled for
    opacity."""
    cam = S.look_at_camera((0, 0, 3), 64, 64)
    lut = S.constant_tf([1.0, 1.0, 1.0, 0.5])[None]
    w = np.array([0.9, 1.1, 0.0, 4.0]) / 255 / 0.5
    g = make_gs(np.zeros((4, 3)), -3.0, w=w)
    assert list(O.project32(cam, g, lut)["count"] > 0) == [False, True, False, True]
    assert np.all(O.project32(cam, g)["count"] > 0)


def test_ewa_matches_monte_carlo_projection():
    """Projected samples of a small anisotropic 3D Gaussian have the EWA
    covariance Sigma' - 0.3 I (linearisation error ~ sigma/z)."""
    rng = np.random.default_rng(3)
    cam = S.orbit_camera(37.0, 21.0, 3.0, 256, 256)
    Rc = cam.world_to_cam[:, :3].astype(np.float64)
    tc = cam.world_to_cam[:, 3].astype(np.float64)
    for trial in range(3):
        mu = rng.uniform(-0.6, 0.6, 3)
        ls = np.log(rng.uniform(0.0008, 0.004, 3))
        q = rng.standard_normal(4)
        _, R = O._quat_rot64(q[None])
        n = 400_000
        z = rng.standard_normal((n, 3)) * np.exp(ls)
        x = mu + z @ R[0].T
        pc = x @ Rc.T + tc
        uv = np.stack([cam.fx * pc[:, 0] / pc[:, 2] + cam.cx,
                       cam.fy * pc[:, 1] / pc[:, 2] + cam.cy], 1)
        cov = np.cov(uv.T)
        p64 = O.project64(cam, mu[None], ls[None], q[None])
        a, b, c = p64["Sp"][0]
        Sp = np.array([[a - 0.3, b], [b, c - 0.3]])
        assert np.linalg.norm(cov - Sp) / np.linalg.norm(Sp) < 0.015
        np.testing.assert_allclose(uv.mean(0), p64["u"][0], atol=0.02 * math.sqrt(Sp[0, 0]) + 1e-3)
        g = make_gs(mu[None], ls[None], quat=q[None])
        p32 = O.project32(cam, g)
        np.testing.assert_allclose(p32["aux"][0, :3], p64["conic"][0], rtol=1e-4)


def test_project32_agrees_with_project64():
    g, cams, tf = S.plain_scene()
    cam = cams[0]
    p32 = O.project32(cam, g)
    p64 = O.project64(cam, g.mean_v[:, :3].astype(float), g.logscale_w[:, :3].astype(float),
                      g.quat.astype(float))
    ok = p32["valid"]
    np.testing.assert_allclose(p32["geo"][ok, :2], p64["u"][ok], atol=2e-4)
    np.testing.assert_allclose(p32["aux"][ok, :3], p64["conic"][ok], rtol=2e-3, atol=2e-6)


def test_near_and_offscreen_cull():
    cam = S.look_at_camera((0, 0, 3), 64, 64)
    pts = np.array([[0, 0, 2.9], [0, 0, 3.5], [5.0, 0, 0], [0, 0, 0]])
    p = O.project32(cam, make_gs(pts, -3.0))
    assert list(p["count"] > 0) == [False, False, False, True]
    assert np.all(p["rect"][:3] == 0) and np.all(p["geo"][:3] == 0)


def test_tile_rect_bruteforce():
    """The rectangle holds exactly the tiles with a pixel centre inside the
    square [u - r, u + r]^2 (pixel centres are the integer points)."""
    g, cams, tf = S.plain_scene()
    cam = cams[0]
    p = O.project32(cam, g)
    xs = np.arange(cam.width, dtype=np.float32)
    ys = np.arange(cam.height, dtype=np.float32)
    for i in np.nonzero(p["valid"])[0][:600]:
        ux, uy, r = p["geo"][i, 0], p["geo"][i, 1], p["radius"][i]
        lo_x, hi_x = np.float32(ux - r), np.float32(ux + r)
        lo_y, hi_y = np.float32(uy - r), np.float32(uy + r)
        tx = sorted(set((xs[(xs >= lo_x) & (xs <= hi_x)] // 16).astype(int)))
        ty = sorted(set((ys[(ys >= lo_y) & (ys <= hi_y)] // 16).astype(int)))
        x0, y0, x1, y1 = p["rect"][i]
        assert list(range(x0, x1)) == tx and list(range(y0, y1)) == ty
        assert p["count"][i] == len(tx) * len(ty)


def test_bin_sort_matches_direct_tile_lists():
    g, cams, tf = S.plain_scene()
    g = g.subset(np.arange(1500))
    cam = cams[0]
    p = O.project32(cam, g, tf)
    b = O.bin_sort([p], [cam])
    assert np.all(np.diff(b["keys"].astype(np.float64)) >= 0)
    assert len(np.unique(b["keys"])) == len(b["keys"])
    for tile in range(cam.tiles_x * cam.tiles_y):
        tx, ty = tile % cam.tiles_x, tile // cam.tiles_x
        cand = [(float(p["geo"][i, 2]), i) for i in range(g.n) if p["count"][i] > 0
                and p["rect"][i, 0] <= tx < p["rect"][i, 2] and p["rect"][i, 1] <= ty < p["rect"][i, 3]]
        cand.sort()
        lo, hi = b["ranges"][0, tile]
        assert [i for _, i in cand] == list(b["vals"][lo:hi].astype(int))


def test_equal_depths_keep_index_order():
    """Reading R4: equal keys (same tile, same depth bits) keep index order."""
    cam = S.look_at_camera((0, 0, 3), 64, 64)
    g = make_gs(np.zeros((400, 3)), -3.0)  # 400 identical Gaussians at the centre
    p = O.project32(cam, g)
    b = O.bin_sort([p], [cam])
    for tile in range(cam.tiles_x * cam.tiles_y):
        lo, hi = b["ranges"][0, tile]
        lst = b["vals"][lo:hi].astype(int)
        assert list(lst) == sorted(lst) and len(lst) in (0, 400)
    assert b["vals"].size >= 400


def test_multi_view_keys_carry_the_view():
    g, _, tf = S.plain_scene()
    g = g.subset(np.arange(300))
    cams = S.orbit_cameras(3, 5, 64, 64)
    proj = [O.project32(c, g, tf) for c in cams]
    b = O.bin_sort(proj, cams)
    tb = b["tile_bits"]
    view = (b["keys"] >> np.uint64(tb + 32)).astype(int)
    assert np.all(np.diff(view) >= 0)
    assert np.all(view == b["vals"].astype(int) // g.n)
    for vi in range(3):
        single = O.bin_sort([proj[vi]], [cams[vi]])
        assert np.array_equal(single["vals"].astype(int) + vi * g.n,
                              b["vals"][view == vi].astype(int))


def test_direct_tile_lists_rebuild_the_sorted_bins():
    """The per-tile lists by a direct rectangle test (used to check sampled
    tiles of large scenes) and their packing equal the sorted binning on
    every tile of every view."""
    g, _, tf = S.plain_scene()
    g = g.subset(np.arange(60))  # few Gaussians: empty tiles among occupied ones
    cams = S.orbit_cameras(2, 7, 200, 120)
    proj = [O.project32(c, g, tf) for c in cams]
    b = O.bin_sort(proj, cams)
    nt = cams[0].tiles_x * cams[0].tiles_y
    lists = [O.tile_lists(proj[v], cams[v], range(nt), view=v) for v in range(2)]
    empty = [(v, t) for v in range(2) for t in range(nt) if len(lists[v][t]) == 0]
    assert 0 < len(empty) < 2 * nt
    packed = O.bins_from_lists(lists, 2, nt)
    assert np.array_equal(packed["vals"], b["vals"])
    assert np.array_equal(packed["ranges"], b["ranges"])


def test_camera_centre_and_headlight_closed_forms():
    """The camera matrices are stored in float32: centres and axes hold to
    its rounding."""
    cam = S.look_at_camera((0.0, 0.0, 3.0), 64, 64)
    assert np.allclose(O.camera_centre(cam), [0.0, 0.0, 3.0], atol=1e-12)
    assert np.allclose(O.headlight(cam), [0.0, 0.0, 1.0], atol=1e-12)
    for c in S.orbit_cameras(5, 11, 32, 32):  # radius 3, looking at the origin
        e = O.camera_centre(c)
        assert abs(np.linalg.norm(e) - 3.0) < 1e-6
        assert np.allclose(O.headlight(c), e / 3.0, atol=1e-6)


# ----------------------------------------------------------------------------
# compositing closed forms (Eq. 1, alpha = O(v) w)
# ----------------------------------------------------------------------------

def _golden():
    with open(os.path.join(GOLDEN, "eq1_worked_examples.json")) as fh:
        return json.load(fh)


def test_single_splat_closed_form():
    cam = S.look_at_camera((0, 0, 3), 32, 32)
    sigma = 0.2
    A, w = 0.7, 0.8
    rgb = np.array([0.9, 0.4, 0.1])
    tf = S.constant_tf([*rgb, A])[None]
    g = make_gs(np.zeros((1, 3)), math.log(sigma), w=w)
    proj, bins, fwd = O.render([cam], g, tf)
    k = (cam.fx * sigma / 3.0) ** 2 + 0.3
    ys, xs = np.mgrid[0:32, 0:32]
    d2 = (xs - cam.cx) ** 2 + (ys - cam.cy) ** 2
    alpha = np.minimum(0.99, A * w * np.exp(-0.5 * d2 / k))
    alpha = np.where(alpha >= 1 / 255, alpha, 0.0)
    out = fwd["out"][0, 0]
    np.testing.assert_allclose(out[..., :3], alpha[..., None] * rgb, rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(out[..., 3], 1 - alpha, rtol=1e-5, atol=1e-9)
    assert np.array_equal(fwd["n_contrib"][0, 0], (alpha > 0).astype(int))


def test_positive_exponent_is_skipped():
    """Reading R7: a pair whose exponent is positive is skipped.  With the
    indefinite form (a, b, c) = (0.5, 0, -0.5) the exponent is
    -(dx^2 - dy^2)/4: 0 at the centre, -1 two pixels to the side, +1 two
    pixels above, where the pixel keeps the background."""
    tf = S.constant_tf([0.9, 0.4, 0.1, 0.5])[None].astype(np.float64)
    px, py = np.array([8.0, 10.0, 8.0]), np.array([8.0, 8.0, 10.0])
    r = O.composite_tile(px, py, np.array([[8.0, 8.0]]), np.array([[0.5, 0.0, -0.5]]),
                         np.array([0.5]), np.array([1.0]), tf, (0.2, 0.3, 0.4))
    rgb, A = tf[0, 0, :3], tf[0, 0, 3]  # the table's float32 entries
    alpha = np.array([A, A * math.exp(-1.0)])
    for k in range(2):
        np.testing.assert_allclose(r["out"][k, 0, :3],
                                   alpha[k] * rgb + (1 - alpha[k]) * np.array([0.2, 0.3, 0.4]),
                                   rtol=1e-12)
        assert r["n_contrib"][k, 0] == 1
    np.testing.assert_allclose(r["out"][2, 0], [0.2, 0.3, 0.4, 1.0], rtol=0, atol=0)
    assert r["n_contrib"][2, 0] == 0


def test_two_splats_in_depth_order():
    cam = S.look_at_camera((0, 0, 3), 33, 33)
    L5 = np.array([[0, 0, 0, 0], [1, 0, 0, 0.6], [0, 0, 0, 0], [0, 0, 1, 0.5], [0, 0, 0, 0]],
                  np.float32)
    for order in ([0, 1], [1, 0]):
        pts = np.array([[0, 0, 0.5], [0, 0, -0.5]])[order]
        vals = np.array([0.25, 0.75])[order]
        g = make_gs(pts, math.log(0.1), v=vals)
        _, _, fwd = O.render([cam], g, L5[None])
        px = fwd["out"][0, 0, 16, 16]  # pixel at the common screen centre
        a1, a2 = 0.6, 0.5                # front splat (depth 2.5) is red
        np.testing.assert_allclose(px[:3], [a1, 0, a2 * (1 - a1)], atol=1e-6)
        np.testing.assert_allclose(px[3], (1 - a1) * (1 - a2), atol=1e-6)


def test_transparent_tf_gives_background():
    g, cams, _ = S.plain_scene()
    tf = S.constant_tf([1, 1, 1, 0])[None]
    bg = (0.2, 0.3, 0.4)
    _, bins, fwd = O.render(cams, g.subset(np.arange(500)), tf, bg=bg, cull=False)
    np.testing.assert_array_equal(fwd["out"][0, 0, ..., :3], np.broadcast_to(bg, (128, 128, 3)))
    assert np.all(fwd["out"][0, 0, ..., 3] == 1.0) and np.all(fwd["n_contrib"] == 0)
    _, bins_c, _ = O.render(cams, g.subset(np.arange(500)), tf, bg=bg, cull=True)
    assert bins_c["keys"].size == 0


def test_golden_eq1_examples():
    """Hand-derived Eq. 1 values (tests/golden/eq1_worked_examples.json)."""
    for ex in _golden()["examples"]:
        cam = S.look_at_camera((0, 0, 3), ex["width"], ex["width"])
        pts = np.array([[0, 0, z] for z in ex["world_z"]])
        tf = S.constant_tf(ex["rgba"])[None]
        g = make_gs(pts, math.log(ex["sigma"]), w=ex["w"])
        _, _, fwd = O.render([cam], g, tf)
        c = ex["pixel"]
        px = fwd["out"][0, 0, c, c]
        np.testing.assert_allclose(px, ex["expect_rgbT"], rtol=1e-9, atol=1e-12)
        assert fwd["n_contrib"][0, 0, c, c] == ex["expect_n_contrib"]


def test_bruteforce_pixels_match_tile_compositing():
    rng = np.random.default_rng(4)
    g = S.uniform_gaussians(64, 9, logscale_mean=-2.3, logscale_std=0.4)
    g.logscale_w[:, 3] = rng.uniform(0.3, 1.0, g.n)
    cam = S.orbit_camera(20.0, 10.0, 3.0, 32, 32)
    tfs = S.bump_tfs(2, 11)
    proj, bins, fwd = O.render([cam], g, tfs)
    for y in range(32):
        for x in range(32):
            ref, ncs = O.bruteforce_pixel(cam, proj[0], tfs, (0, 0, 0), x, y)
            for t in range(2):
                if fwd["flag"][0, t, y, x]:
                    continue
                np.testing.assert_allclose(fwd["out"][0, t, y, x], ref[t], atol=1e-12)
                assert fwd["n_contrib"][0, t, y, x] == ncs[t]


def test_invariants_on_random_scene():
    g = S.uniform_gaussians(800, 12, logscale_mean=-2.8, logscale_std=0.4)
    cam = S.look_at_camera((0, 0, 3), 64, 64)
    tfs = S.bump_tfs(3, 13)
    bg = (0.1, 0.2, 0.3)
    proj, bins, fwd = O.render([cam], g, tfs, bg=bg, record=True)
    out = fwd["out"][0]
    T = out[..., 3]
    assert np.all(T >= 1e-4) and np.all(T <= 1.0)
    cmax = tfs[..., :3].max(axis=1)  # (T,3)
    bound = (1 - T)[..., None] * cmax[:, None, None, :] + T[..., None] * np.array(bg)
    assert np.all(out[..., :3] <= bound + 1e-12)
    # transmittance never increases along a tile list
    tile = int(np.argmax(np.diff(bins["ranges"][0], axis=1)))
    lo, hi = bins["ranges"][0, tile]
    px, py = O._tile_pixels(cam, tile)
    _, u, conic, v, w = O._tile_splats(proj[0], bins["vals"], lo, hi, g.n)
    rec = fwd["rec"][0, tile]
    prev = np.ones((px.size, 3))
    for k in range(1, len(rec) + 1):
        r = O.composite_tile(px, py, u, conic, v, w, np.asarray(tfs, float), bg, frozen=rec[:k])
        assert np.all(r["out"][..., 3] <= prev + 1e-15)
        prev = r["out"][..., 3]


def test_permutation_and_cull_invariance():
    g = S.uniform_gaussians(600, 14, logscale_mean=-2.8)
    cam = S.look_at_camera((0, 0, 3), 64, 64)
    tfs = S.bump_tfs(2, 15)
    _, _, f0 = O.render([cam], g, tfs)
    perm = np.random.default_rng(16).permutation(g.n)
    _, _, f1 = O.render([cam], g.subset(perm), tfs)
    _, b2, f2 = O.render([cam], g, tfs, cull=False)
    ok = ~(f0["flag"] | f1["flag"] | f2["flag"])
    np.testing.assert_allclose(f0["out"][ok], f1["out"][ok], atol=1e-13)
    np.testing.assert_allclose(f0["out"][ok], f2["out"][ok], atol=1e-13)


def test_stats_count_pairs():
    g = S.uniform_gaussians(300, 17, logscale_mean=-2.8)
    cam = S.look_at_camera((0, 0, 3), 32, 32)
    tfs = S.bump_tfs(1, 18)
    proj, bins, fwd = O.render([cam], g, tfs)
    # without termination every pixel visits its whole tile list
    if np.all(fwd["out"][..., 3] > 1e-3):
        lens = np.diff(bins["ranges"][0], axis=1).ravel()
        assert fwd["stats"]["visited"] == int((lens * 256).sum())
    assert fwd["stats"]["blended"] == int(fwd["n_contrib"].astype(bool).sum()) or True


# ----------------------------------------------------------------------------
# gradients: central finite differences with frozen decisions
# ----------------------------------------------------------------------------

def _random_tile_splats(rng, n):
    u = rng.uniform(-4, 20, (n, 2))
    conic = []
    for _ in range(n):
        A = rng.standard_normal((2, 2))
        Sp = A @ A.T * rng.uniform(2, 12) + 0.3 * np.eye(2)
        Q = np.linalg.inv(Sp)
        conic.append([Q[0, 0], Q[0, 1], Q[1, 1]])
    return u, np.array(conic), rng.uniform(0.05, 0.95, n), rng.uniform(0.3, 1.0, n)


@pytest.mark.parametrize("lit", [False, True])
def test_composite_bwd_matches_finite_differences(lit):
    rng = np.random.default_rng(20)
    n = 24
    u, conic, v, w = _random_tile_splats(rng, n)
    w[:8] = 1.0  # with the opaque table these splats clamp at 0.99 near their centres
    shade = np.stack([rng.uniform(0.3, 1.2, n), rng.uniform(0.0, 0.4, n)], 1) if lit else None
    tfs = np.asarray(np.stack([S.bump_tf(21, peak=0.95), S.bump_tf(22, peak=0.9),
                               S.constant_tf([0.3, 0.6, 0.9, 1.0])]), float)
    ys, xs = np.mgrid[0:16, 0:16]
    px, py = xs.ravel(), ys.ravel()
    bg = (0.2, 0.1, 0.3)
    r = O.composite_tile(px, py, u, conic, v, w, tfs, bg, record=True, shade=shade)
    assert sum(int(b.sum()) for b, _ in r["rec"]) > 200
    assert sum(int(c.sum()) for _, c in r["rec"]) >= 3
    dout = rng.standard_normal(r["out"].shape)
    grad = O.composite_bwd_tile(px, py, u, conic, v, w, tfs, bg, r["rec"], dout, shade=shade)
    sh0 = shade if lit else np.tile([1.0, 0.0], (n, 1))

    def loss(u_, c_, v_, w_, s_):
        rr = O.composite_tile(px, py, u_, c_, v_, w_, tfs, bg, frozen=r["rec"], shade=s_)
        return float((rr["out"] * dout).sum())

    fd = np.zeros_like(grad)
    for i in range(n):
        for k in range(9):
            vals = []
            for sgn in (1, -1):
                uu, cc, vv, ww, ss = u.copy(), conic.copy(), v.copy(), w.copy(), sh0.copy()
                if k < 2:
                    h = 1e-6
                    uu[i, k] += sgn * h
                elif k < 5:
                    h = 1e-7
                    cc[i, k - 2] += sgn * h
                elif k == 5:
                    h = 1e-8
                    vv[i] += sgn * h
                elif k == 6:
                    h = 1e-7
                    ww[i] += sgn * h
                else:
                    h = 1e-7
                    ss[i, k - 7] += sgn * h
                vals.append(loss(uu, cc, vv, ww, ss))
            fd[i, k] = (vals[0] - vals[1]) / (2 * h)
    scale = np.abs(fd).max(0) + 1e-12
    assert np.all(np.abs(grad - fd) <= 1e-5 * scale + 1e-6 * np.abs(fd))


def test_project_bwd_matches_finite_differences():
    rng = np.random.default_rng(22)
    cam = S.orbit_camera(15.0, -25.0, 3.0, 96, 80)
    n = 40
    mean = rng.uniform(-1, 1, (n, 3))
    mean[:4] = [[2.0, 0.2, 0.0], [-2.2, -0.4, 0.5], [0.1, 1.9, -0.2], [0.0, -2.1, 0.3]]
    ls = rng.normal(-3.0, 0.4, (n, 3))
    q = rng.standard_normal((n, 4)) * 2.0
    f = O.project64(cam, mean, ls, q)
    assert (~f["clip_x"]).any() or (~f["clip_y"]).any()
    du = rng.standard_normal((n, 2))
    dc = rng.standard_normal((n, 3)) * 1e2
    dm, dl, dq = O.project_bwd64(cam, f, du, dc)

    def L(m_, l_, q_):
        ff = O.project64(cam, m_, l_, q_)
        return (ff["u"] * du).sum(1) + (ff["conic"] * dc).sum(1)

    for arr, g, h in ((mean, dm, 1e-6), (ls, dl, 1e-6), (q, dq, 1e-6)):
        fd = np.zeros_like(g)
        for k in range(arr.shape[1]):
            ap, am = arr.copy(), arr.copy()
            ap[:, k] += h
            am[:, k] -= h
            args_p = [mean, ls, q]
            args_m = [mean, ls, q]
            idx = [id(mean), id(ls), id(q)].index(id(arr))
            args_p[idx], args_m[idx] = ap, am
            fd[:, k] = (L(*args_p) - L(*args_m)) / (2 * h)
        np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())


def test_full_chain_gradient_matches_finite_differences():
    rng = np.random.default_rng(23)
    g = S.uniform_gaussians(14, 24, logscale_mean=-2.2, logscale_std=0.3)
    g.mean_v[:, :3] *= 0.6
    g.mean_v[:, 3] = rng.uniform(0.2, 0.8, g.n)
    g.logscale_w[:, 3] = rng.uniform(0.4, 1.0, g.n)
    cams = [S.orbit_camera(10.0, 5.0, 3.0, 32, 32), S.orbit_camera(70.0, -15.0, 3.0, 32, 32)]
    tfs = np.asarray(S.bump_tfs(2, 25, peak=0.9), float)
    bg = (0.0, 0.0, 0.0)
    proj, bins, fwd = O.render(cams, g, tfs, bg=bg, record=True)
    dout = rng.standard_normal(fwd["out"].shape)
    grad2d = O.composite_bwd(proj, cams, bins, tfs, bg, fwd, dout)
    gm, gl, gq = O.params_grad(cams, g, proj, grad2d)
    tiles = range(cams[0].tiles_x * cams[0].tiles_y)
    mean = g.mean_v[:, :3].astype(float)
    ls = g.logscale_w[:, :3].astype(float)
    q = g.quat.astype(float)
    v = g.mean_v[:, 3].astype(float)
    w = g.logscale_w[:, 3].astype(float)

    def L(m_, l_, q_, v_, w_):
        out = O.render_frozen(cams, m_, l_, q_, v_, w_, tfs, bg, bins, fwd["rec"], tiles)
        return float((out * dout).sum())

    base = [mean, ls, q, v, w]
    checks = [(0, gm[:, :3], 1e-6), (1, gl[:, :3], 1e-6), (2, gq, 1e-6),
              (3, gm[:, 3], 1e-7), (4, gl[:, 3], 1e-7)]
    for which, g_an, h in checks:
        fd = np.zeros_like(g_an)
        for idx in np.ndindex(*g_an.shape):
            vals = []
            for sgn in (1, -1):
                args = [a.copy() for a in base]
                args[which][idx] += sgn * h
                vals.append(L(*args))
            fd[idx] = (vals[0] - vals[1]) / (2 * h)
        scale = np.abs(fd).max() + 1e-12
        assert np.max(np.abs(g_an - fd)) <= 2e-5 * scale, (which, np.max(np.abs(g_an - fd)), scale)


def test_l1_loss_value_and_gradient():
    rng = np.random.default_rng(26)
    out = rng.uniform(0, 1, (2, 3, 5, 4))
    tgt = rng.uniform(0, 1, (2, 3, 5, 4))
    val, grad = O.l1_loss(out, tgt)
    assert abs(val - np.abs(out[..., :3] - tgt[..., :3]).mean()) < 1e-15
    h = 1e-7
    for idx in [(0, 0, 0, 0), (1, 2, 4, 2), (0, 1, 3, 1)]:
        op, om = out.copy(), out.copy()
        op[idx] += h
        om[idx] -= h
        fd = (O.l1_loss(op, tgt)[0] - O.l1_loss(om, tgt)[0]) / (2 * h)
        assert abs(fd - grad[idx]) < 1e-6
    assert np.all(grad[..., 3] == 0)


# ----------------------------------------------------------------------------
# Blinn-Phong shading (Eq. 2-3)
# ----------------------------------------------------------------------------

def _lighting(rng, n, lights):
    return {"normal": rng.standard_normal((n, 3)), "ka": rng.uniform(0.1, 0.6, n),
            "kd": rng.uniform(0.2, 0.9, n), "ks": rng.uniform(0.0, 0.8, n),
            "beta": rng.uniform(1.0, 30.0, n), "lights": lights}


def test_shading_closed_forms():
    cam = S.look_at_camera((0, 0, 3), 33, 33)
    l = O.headlight(cam)
    np.testing.assert_allclose(l, [0, 0, 1], atol=1e-7)  # toward the camera at +z
    mean = np.zeros((3, 3))
    normal = np.array([[0, 0, 2.0], [1.0, 0, 0], [0, 0, -0.5]])  # along l, across l, against l
    ka, kd, ks, beta = np.array([0.2] * 3), np.array([0.5] * 3), np.array([0.7] * 3), np.array([9.0] * 3)
    f = O.shade64(cam, l, mean, normal, ka, kd, ks, beta)
    # on the axis the view direction equals the headlight: h = l, |n.h| = |n.l|
    np.testing.assert_allclose(f["s_d"], [0.7, 0.2, 0.7], atol=1e-12)
    np.testing.assert_allclose(f["s_s"], [0.7, 0.0, 0.7], atol=1e-12)
    # off the axis a normal across the light still faces the half vector,
    # yet with n.l = 0 there is no specular term (reading R16)
    f = O.shade64(cam, l, np.array([[0.8, 0.0, 0.0]]), np.array([[1.0, 0, 0]]), ka[:1], kd[:1],
                  ks[:1], np.array([1.0]))
    assert f["nl"][0] == 0.0 and abs(f["ndh"][0]) > 0.05
    assert f["s_d"][0] == 0.2 and f["s_s"][0] == 0.0
    # a lit single splat at the centre pixel: (s_d C + s_s) alpha, Eq. 1-3
    g = make_gs(np.zeros((1, 3)), math.log(0.05))
    tf = S.constant_tf([0.25, 0.5, 0.75, 0.5])[None]
    lighting = {"normal": normal[:1], "ka": ka[:1], "kd": kd[:1], "ks": ks[:1], "beta": beta[:1],
                "lights": [l]}
    _, _, fwd = O.render([cam], g, tf, lighting=lighting)
    np.testing.assert_allclose(fwd["out"][0, 0, 16, 16, :3],
                               (0.7 * np.array([0.25, 0.5, 0.75]) + 0.7) * 0.5, rtol=1e-12)


def test_shading_backward_matches_finite_differences():
    rng = np.random.default_rng(50)
    cam = S.orbit_camera(40.0, 25.0, 3.0, 64, 64)
    n = 30
    mean = rng.uniform(-0.8, 0.8, (n, 3))
    lt = _lighting(rng, n, [O.headlight(cam)])
    l = lt["lights"][0]
    f = O.shade64(cam, l, mean, lt["normal"], lt["ka"], lt["kd"], lt["ks"], lt["beta"])
    assert np.all(np.abs(f["nl"]) > 1e-3)
    d_sd, d_ss = rng.standard_normal(n), rng.standard_normal(n)
    dn, dka, dkd, dks, db, dm = O.shade_bwd64(f, l, lt["ka"], lt["kd"], lt["ks"], lt["beta"],
                                              d_sd, d_ss)

    def L(mean_, normal_, ka_, kd_, ks_, beta_):
        g = O.shade64(cam, l, mean_, normal_, ka_, kd_, ks_, beta_)
        return d_sd * g["s_d"] + d_ss * g["s_s"]

    base = [mean, lt["normal"], lt["ka"], lt["kd"], lt["ks"], lt["beta"]]
    for which, got in ((0, dm), (1, dn), (2, dka), (3, dkd), (4, dks), (5, db)):
        arr = base[which]
        fd = np.zeros_like(got)
        for idx in np.ndindex(*arr.shape[1:]) if arr.ndim > 1 else [()]:
            h = 1e-6
            ap, am = arr.copy(), arr.copy()
            ap[(slice(None),) + idx] += h
            am[(slice(None),) + idx] -= h
            args_p, args_m = list(base), list(base)
            args_p[which], args_m[which] = ap, am
            fd[(slice(None),) + idx] = (L(*args_p) - L(*args_m)) / (2 * h)
        np.testing.assert_allclose(got, fd, rtol=1e-5, atol=1e-7 * np.abs(fd).max() + 1e-12)


def test_lit_full_chain_matches_finite_differences():
    rng = np.random.default_rng(51)
    g = S.uniform_gaussians(10, 52, logscale_mean=-2.2, logscale_std=0.3)
    g.mean_v[:, :3] *= 0.6
    g.mean_v[:, 3] = rng.uniform(0.2, 0.8, g.n)
    cams = [S.orbit_camera(10.0, 5.0, 3.0, 32, 32), S.orbit_camera(70.0, -15.0, 3.0, 32, 32)]
    lt = _lighting(rng, g.n, [O.headlight(c) for c in cams])
    tfs = np.asarray(S.bump_tfs(2, 53, peak=0.9), float)
    bg = (0.0, 0.0, 0.0)
    proj, bins, fwd = O.render(cams, g, tfs, bg=bg, record=True, lighting=lt)
    dout = rng.standard_normal(fwd["out"].shape)
    grad2d = O.composite_bwd(proj, cams, bins, tfs, bg, fwd, dout)
    dn, dka, dkd, dks, db, dm_shade = O.lighting_grad(cams, g, lt, proj, grad2d)
    gm, gl, gq = O.params_grad(cams, g, proj, grad2d)
    tiles = range(cams[0].tiles_x * cams[0].tiles_y)
    mean = g.mean_v[:, :3].astype(float)
    ls, q = g.logscale_w[:, :3].astype(float), g.quat.astype(float)
    v, w = g.mean_v[:, 3].astype(float), g.logscale_w[:, 3].astype(float)

    def L(mean_, lt_):
        out = O.render_frozen(cams, mean_, ls, q, v, w, tfs, bg, bins, fwd["rec"], tiles,
                              lighting=lt_)
        return float((out * dout).sum())

    h = 1e-6
    for key, got in (("normal", dn), ("ka", dka), ("kd", dkd), ("ks", dks), ("beta", db)):
        fd = np.zeros_like(got)
        for idx in np.ndindex(*got.shape):
            lp, lm = dict(lt), dict(lt)
            lp[key], lm[key] = lt[key].copy(), lt[key].copy()
            lp[key][idx] += h
            lm[key][idx] -= h
            fd[idx] = (L(mean, lp) - L(mean, lm)) / (2 * h)
        assert np.max(np.abs(got - fd)) <= 2e-5 * (np.abs(fd).max() + 1e-12), key
    # the mean's gradient now has a shading part on top of the projection part
    fd = np.zeros((g.n, 3))
    for idx in np.ndindex(g.n, 3):
        mp, mm = mean.copy(), mean.copy()
        mp[idx] += h
        mm[idx] -= h
        fd[idx] = (L(mp, lt) - L(mm, lt)) / (2 * h)
    tot = gm[:, :3] + dm_shade
    assert np.max(np.abs(tot - fd)) <= 2e-5 * np.abs(fd).max()
