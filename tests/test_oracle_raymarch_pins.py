"""Pins of the raymarching oracle (no GPU).

Trilinear interpolation against linear fields (exact) and scipy's
map_coordinates; box clipping against hand-computed intervals; the
emission-absorption transmittance and colour of a constant medium in closed
form; the early stop; Blinn-Phong shading of a linear field in closed form;
empty volumes; multi-table consistency.
"""
import math

import numpy as np
import pytest
from scipy import ndimage as ndi

from oracle import veg_raymarch_oracle as RM
from paper_2504_13339_gb300 import scenes as S


def grid(R):
    return np.linspace(-1.0, 1.0, R)


def linear_volume(R, a, b, c, e):
    x = grid(R)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return a * X + b * Y + c * Z + e


def test_trilinear_exact_on_linear_fields_and_matches_scipy():
    rng = np.random.default_rng(0)
    R = 9
    a, b, c, e = 0.3, -0.7, 0.2, 0.5
    vol = linear_volume(R, a, b, c, e)
    for p in rng.uniform(-1, 1, (50, 3)):
        v, g = RM.trilinear(vol, p)
        assert v == pytest.approx(a * p[0] + b * p[1] + c * p[2] + e, abs=1e-12)
        assert np.allclose(g, [a, b, c], atol=1e-12)
    rnd = rng.uniform(0, 1, (R, R, R))
    h = 2.0 / (R - 1)
    pts = rng.uniform(-1, 1, (200, 3))
    coords = ((pts + 1.0) / h)[:, ::-1].T  # (z, y, x) index coordinates
    ref = ndi.map_coordinates(rnd, coords, order=1)
    got = np.array([RM.trilinear(rnd, p)[0] for p in pts])
    assert np.allclose(got, ref, atol=1e-12)


def test_vertex_gradients_closed_forms():
    """Central differences are exact for quadratics inside (2x for x^2);
    the one-sided boundary difference of x^2 is x0 + x1."""
    R = 11
    x = grid(R)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    g = RM.vertex_gradients(X * X + 3 * Y - Z * Z * 0.5)
    assert np.allclose(g[:, :, 1:-1, 0], 2 * X[:, :, 1:-1], atol=1e-12)
    assert np.allclose(g[:, :, 0, 0], x[0] + x[1], atol=1e-12)
    assert np.allclose(g[:, :, -1, 0], x[-1] + x[-2], atol=1e-12)
    assert np.allclose(g[..., 1], 3.0, atol=1e-12)
    assert np.allclose(g[1:-1, :, :, 2], -Z[1:-1], atol=1e-12)
    # interpolated gradients are continuous across a cell face
    vol = np.random.default_rng(2).uniform(0, 1, (R, R, R))
    face = -1.0 + 2.0 * 4 / (R - 1)
    a = RM.trilinear(vol, [face - 1e-9, 0.13, -0.4])[1]
    b = RM.trilinear(vol, [face + 1e-9, 0.13, -0.4])[1]
    assert np.allclose(a, b, atol=1e-6)


def test_box_clipping():
    cam = S.look_at_camera((0.0, 0.0, 3.0), 33, 33)
    eye, d = RM.camera_ray(cam, 16, 16)  # the centre pixel looks at the origin
    assert np.allclose(d, [0, 0, -1])
    assert np.allclose(RM.clip_box(eye, d, cam.near), (2.0, 4.0))
    assert RM.clip_box(eye, -d, cam.near) is None
    # a ray passing beside the box misses it
    assert RM.clip_box(np.array([0.0, 1.5, 3.0]), np.array([0.0, 0.0, -1.0]), 0.2) is None


def test_constant_medium_closed_form():
    """v = 0.5 everywhere, a constant table (rgb, A), no shading: n equal
    samples of alpha = 1 - (1-A)^(Delta/h), so T = (1-alpha)^n and
    C = rgb (1 - T) + T bg."""
    R = 17
    vol = np.full((R, R, R), 0.5)
    lut = S.constant_tf([0.9, 0.4, 0.1, 0.05]).astype(np.float64)[None]
    rgb, A = lut[0, 0, :3], lut[0, 0, 3]  # the table's float32 values
    cam = S.look_at_camera((0.0, 0.0, 3.0), 33, 33)
    h = 2.0 / (R - 1)
    step = h / 2
    bg = (0.2, 0.3, 0.4)
    out, flag = RM.march_pixel(cam, vol, lut, 16, 16, step, None, bg)
    n = math.floor(2.0 / step)
    alpha = 1.0 - (1.0 - A) ** (step / h)
    T = (1.0 - alpha) ** n
    assert out[0, 3] == pytest.approx(T, rel=1e-12)
    assert np.allclose(out[0, :3], rgb * (1 - T) + T * np.array(bg), rtol=1e-12)
    # the step size does not change the medium: T -> (1 - A)^(L/h)
    out2, _ = RM.march_pixel(cam, vol, lut, 16, 16, h / 8, None, bg)
    assert out2[0, 3] == pytest.approx((1 - A) ** (2.0 / h), rel=1e-9)


def test_early_stop_after_crossing():
    R = 9
    vol = np.full((R, R, R), 0.5)
    lut = S.constant_tf([1.0, 1.0, 1.0, 0.85]).astype(np.float64)[None]
    cam = S.look_at_camera((0.0, 0.0, 3.0), 33, 33)
    h = 2.0 / (R - 1)
    out, _ = RM.march_pixel(cam, vol, lut, 16, 16, h / 2, None)
    alpha = 1.0 - (1.0 - lut[0, 0, 3]) ** 0.5
    k = 1
    while (1 - alpha) ** k >= RM.T_STOP:  # samples until T falls below 1e-4
        k += 1
    assert k < 2.0 / (h / 2)  # stops inside the box
    assert out[0, 3] == pytest.approx((1 - alpha) ** k, rel=1e-12)
    assert out[0, 3] < RM.T_STOP <= out[0, 3] / (1 - alpha)


def test_shading_of_a_linear_field_closed_form():
    """v = 0.3 x + 0.5 has the gradient (0.3, 0, 0) everywhere: every sample
    has the normal -x, so its colour is (k_a + k_d |n.l|) C + k_s |n.h|^beta."""
    R = 17
    vol = linear_volume(R, 0.3, 0.0, 0.0, 0.5)
    lut = S.constant_tf([0.2, 0.6, 0.9, 0.02]).astype(np.float64)[None]
    rgb = lut[0, 0, :3]
    cam = S.orbit_camera(35.0, 20.0, 3.0, 41, 41)
    mat = (0.3, 0.6, 0.25, 12.0)
    i, j = 8, 29  # off the optical axis: the view and light directions differ
    out, _ = RM.march_pixel(cam, vol, lut, i, j, 1.0 / 16, mat)
    eye, d = RM.camera_ray(cam, i, j)
    light = -np.asarray(cam.world_to_cam, np.float64)[2, :3]
    n = np.array([-1.0, 0.0, 0.0])
    hv = (-d + light) / np.linalg.norm(-d + light)
    c = (mat[0] + mat[1] * abs(n @ light)) * rgb + mat[2] * abs(n @ hv) ** mat[3]
    T = out[0, 3]
    assert 0.05 < T < 0.95
    assert np.allclose(out[0, :3], c * (1 - T), rtol=1e-12)


def test_sample_positions_closed_form():
    """v = 0.5 + 0.4 z seen along the z axis through a table that is exactly
    linear (opacity 0.02 + 0.1 v, grey level v): sample k sits at
    z_k = 1 - (k + 1/2) Delta, so every sample's alpha and colour is known
    and the composite is a short explicit product."""
    R = 17
    vol = linear_volume(R, 0.0, 0.0, 0.4, 0.5)
    x = np.arange(256) / 255
    lut = np.stack([x, x, x, 0.02 + 0.1 * x], 1)[None]
    cam = S.look_at_camera((0.0, 0.0, 3.0), 33, 33)
    h = 2.0 / (R - 1)
    step = 0.1
    out, _ = RM.march_pixel(cam, vol, lut, 16, 16, step, None)
    C, T = 0.0, 1.0
    for k in range(20):  # L = 2, 2 / 0.1 = 20 samples
        v = 0.5 + 0.4 * (1.0 - (k + 0.5) * step)
        a = 1.0 - (1.0 - (0.02 + 0.1 * v)) ** (step / h)
        C += T * a * v
        T *= 1.0 - a
    assert out[0, 3] == pytest.approx(T, rel=1e-12)
    assert out[0, 0] == pytest.approx(C, rel=1e-12)


def test_flat_volume_keeps_only_the_ambient_term():
    """A constant volume has no gradient, hence no normal: every shaded
    sample has the colour k_a C."""
    R = 9
    vol = np.full((R, R, R), 0.5)
    lut = S.constant_tf([0.9, 0.4, 0.1, 0.05]).astype(np.float64)[None]
    cam = S.look_at_camera((0.0, 0.0, 3.0), 33, 33)
    plain, _ = RM.march_pixel(cam, vol, lut, 10, 20, 0.05, None)
    lit, _ = RM.march_pixel(cam, vol, lut, 10, 20, 0.05, (0.3, 0.6, 0.2, 8.0))
    assert lit[0, 3] == plain[0, 3]
    assert np.allclose(lit[0, :3], 0.3 * plain[0, :3], rtol=1e-12)


def test_empty_volume_and_multi_table_consistency():
    R = 9
    rng = np.random.default_rng(1)
    vol = rng.uniform(0, 1, (R, R, R))
    cam = S.look_at_camera((0.0, 0.0, 3.0), 12, 10)
    empty = S.constant_tf([1, 1, 1, 0]).astype(np.float64)[None]
    out, _ = RM.render(cam, vol, empty, 0.1, bg=(0.1, 0.2, 0.3))
    assert np.allclose(out[..., :3], [0.1, 0.2, 0.3]) and np.all(out[..., 3] == 1.0)
    tfs = S.bump_tfs(2, 5).astype(np.float64)
    mat = (0.3, 0.6, 0.2, 10.0)
    both, _ = RM.render(cam, vol, tfs, 0.05, mat)
    for t in range(2):
        one, _ = RM.render(cam, vol, tfs[t:t + 1], 0.05, mat)
        assert np.array_equal(both[t], one[0])


def test_table_lookup_closed_forms():
    """Linear interpolation over [0, 1] (reading R6): a linear table gives
    the linear function, a random table agrees with numpy's interpolation,
    table nodes are hit exactly, values outside [0, 1] clamp to the end
    entries, and v = 1 takes the last entry."""
    for L in (2, 3, 256, 4096):
        c = np.array([0.25, -1.5, 3.0, 0.75])
        lut = np.arange(L)[:, None] / (L - 1) * c[None]
        for v in np.random.default_rng(L).uniform(0.0, 1.0, 50):
            assert np.allclose(RM.tf_lookup(lut, v), v * c, rtol=0, atol=1e-12)
        rnd = np.random.default_rng(L + 1).standard_normal((L, 4))
        xk = np.arange(L) / (L - 1)
        for v in np.random.default_rng(L + 2).uniform(0.0, 1.0, 50):  # numpy's interpolation
            ref = [np.interp(v, xk, rnd[:, c]) for c in range(4)]
            assert np.allclose(RM.tf_lookup(rnd, v), ref, rtol=0, atol=1e-12)
        for k in range(0, L, max(1, L // 7)):
            assert np.array_equal(RM.tf_lookup(rnd, k / (L - 1)), rnd[k])
        assert np.array_equal(RM.tf_lookup(rnd, -0.3), rnd[0])
        assert np.array_equal(RM.tf_lookup(rnd, 1.0), rnd[-1])
        assert np.array_equal(RM.tf_lookup(rnd, 7.0), rnd[-1])


def test_camera_ray_reprojects_to_its_pixel():
    """A point on the ray of pixel (i, j) projects back to (i, j) on a
    non-square image (x = i along the width, y = j along the height), and the
    ray starts at the camera centre."""
    cam = S.orbit_camera(40.0, 15.0, 3.0, 61, 23)
    w2c = np.asarray(cam.world_to_cam, np.float64)
    for i, j in ((3, 17), (50, 2), (30, 11)):
        eye, d = RM.camera_ray(cam, i, j)
        assert abs(np.linalg.norm(d) - 1.0) < 1e-12
        assert np.allclose(w2c[:, :3] @ eye + w2c[:, 3], 0.0, atol=1e-6)
        c = w2c[:, :3] @ (eye + 2.5 * d) + w2c[:, 3]
        assert c[2] > 0
        # to 1e-4 px: the stored rotation is float32, so its transpose is
        # its inverse only to that rounding
        assert abs(cam.fx * c[0] / c[2] + cam.cx - i) < 1e-4
        assert abs(cam.fy * c[1] / c[2] + cam.cy - j) < 1e-4


def test_trilinear_hits_vertices_on_every_face():
    """At vertex positions, including those on the upper faces x, y or z = 1
    (where the cell index is clamped), the value is the vertex value."""
    R = 6
    vol = np.random.default_rng(5).uniform(0.0, 1.0, (R, R, R))
    x = grid(R)
    for zi, yi, xi in ((R - 1, 2, 3), (1, R - 1, 4), (2, 3, R - 1), (R - 1, R - 1, R - 1),
                       (0, 0, 0), (3, 1, 2)):
        val, _ = RM.trilinear(vol, (x[xi], x[yi], x[zi]))
        assert val == pytest.approx(vol[zi, yi, xi], abs=1e-12)


def test_sample_count_of_a_fractional_segment():
    """With the box crossing 2 long and Delta = 0.15 the ray takes
    floor(2 / 0.15) = 13 samples at z_k = 1 - (k + 1/2) Delta."""
    R = 17
    vol = linear_volume(R, 0.0, 0.0, 0.4, 0.5)
    x = np.arange(256) / 255
    lut = np.stack([x, x, x, 0.02 + 0.1 * x], 1)[None]
    cam = S.look_at_camera((0.0, 0.0, 3.0), 33, 33)
    h = 2.0 / (R - 1)
    step = 0.15
    out, _ = RM.march_pixel(cam, vol, lut, 16, 16, step, None)
    C, T = 0.0, 1.0
    for k in range(13):
        v = 0.5 + 0.4 * (1.0 - (k + 0.5) * step)
        a = 1.0 - (1.0 - (0.02 + 0.1 * v)) ** (step / h)
        C += T * a * v
        T *= 1.0 - a
    assert out[0, 3] == pytest.approx(T, rel=1e-12)
    assert out[0, 0] == pytest.approx(C, rel=1e-12)


def test_no_specular_where_the_light_is_tangent():
    """v = 0.3 x + 0.5 seen from (0, 0, 3): the normal -x is perpendicular
    to the headlight (+z), so diffuse and specular vanish (reading R27) even
    off axis, where n.h is not zero, and the colour is k_a C."""
    R = 17
    vol = linear_volume(R, 0.3, 0.0, 0.0, 0.5)
    lut = S.constant_tf([0.2, 0.6, 0.9, 0.02]).astype(np.float64)[None]
    cam = S.look_at_camera((0.0, 0.0, 3.0), 41, 41)
    i, j = 5, 30
    _, d = RM.camera_ray(cam, i, j)
    light = -np.asarray(cam.world_to_cam, np.float64)[2, :3]
    hv = (-d + light) / np.linalg.norm(-d + light)
    assert abs(np.array([-1.0, 0, 0]) @ hv) > 0.05
    plain, _ = RM.march_pixel(cam, vol, lut, i, j, 1.0 / 16, None)
    lit, _ = RM.march_pixel(cam, vol, lut, i, j, 1.0 / 16, (0.3, 0.6, 0.25, 1.0))
    assert lit[0, 3] == plain[0, 3]
    assert np.allclose(lit[0, :3], 0.3 * plain[0, :3], rtol=1e-12, atol=0.0)
