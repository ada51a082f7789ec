"""The seeded synthetic inputs follow their stated recipe (no GPU): the
plain scene's distributions, the blob-field sampling and its scalars, the
log-scales of half the mean spacing, the perturbed target copy, the bump
tables and the camera's field of view."""
import math

import numpy as np

from paper_2504_13339_gb300 import scenes as S


def test_plain_scene_distributions_and_seeding():
    g, cams, tfs = S.plain_scene()
    g2, _, tfs2 = S.plain_scene()
    assert np.array_equal(g.mean_v, g2.mean_v) and np.array_equal(tfs, tfs2)
    assert g.n == 4096
    mu = g.mean_v[:, :3].astype(np.float64)
    assert np.all(np.abs(mu) <= 1.0)
    assert np.all(np.abs(mu.mean(0)) < 0.05) and np.all(np.abs(mu.var(0) - 1 / 3) < 0.03)
    ls = g.logscale_w[:, :3].astype(np.float64)
    assert abs(ls.mean() + 3.5) < 0.02 and abs(ls.std() - 0.3) < 0.02
    v = g.mean_v[:, 3]
    assert v.min() >= 0.0 and v.max() <= 1.0 and abs(v.mean() - 0.5) < 0.03
    assert np.all(g.logscale_w[:, 3] == 1.0)
    assert np.allclose(np.linalg.norm(g.quat.astype(np.float64), axis=1), 1.0, atol=1e-6)
    cam = cams[0]
    assert (cam.width, cam.height) == (128, 128)
    f = 64.0 / math.tan(math.radians(22.5))  # fov 45 degrees over 128 pixels
    assert abs(cam.fx - f) < 1e-3 and abs(cam.fy - f) < 1e-3
    assert tfs.shape == (1, 256, 4)


def test_bump_tables():
    for seed in range(20):
        t = S.bump_tf(seed)
        assert t.shape == (256, 4) and t.dtype == np.float32
        assert np.all((t[:, :3] >= 0.0) & (t[:, :3] <= 1.0))
        # three bumps of peak 0.8 and width >= 0.03: a table node lies within
        # half a spacing of each centre, so the largest entry is near 0.8
        assert 0.79 < t[:, 3].max() <= 0.8 + 1e-7 and t[:, 3].min() >= 0.0


def test_blob_field_sampling_scalars_and_scales():
    n = 20000
    g, bf = S.field_gaussians(n, 8, 3)
    mu = g.mean_v[:, :3].astype(np.float64)
    assert np.all(np.abs(mu) <= 1.0)
    f = bf.value(mu)
    assert np.allclose(g.mean_v[:, 3], np.clip(f / f.max(), 0, 1), atol=1e-6)
    assert g.mean_v[:, 3].max() == 1.0
    # means follow the density: the field is far larger at the samples than
    # at uniform points of the cube
    u = np.random.default_rng(0).uniform(-1.0, 1.0, (n, 3))
    assert f.mean() > 2.0 * bf.value(u).mean()
    ls = g.logscale_w[:, :3].astype(np.float64)
    assert abs(ls.mean() - math.log(1.0 / n ** (1 / 3))) < 0.02  # half the mean spacing
    assert np.all(bf.amp >= 0.3) and np.all(bf.amp <= 1.0)
    assert np.all(np.abs(bf.center) <= 0.7)
    assert np.all((bf.sigma >= 0.08) & (bf.sigma <= 0.35))
    for r in bf.rot:
        assert np.allclose(r @ r.T, np.eye(3), atol=1e-12) and np.linalg.det(r) > 0


def test_perturbed_target_copy():
    g, _ = S.field_gaussians(20000, 8, 4)
    t = S.perturbed(g, 5)
    dm = (t.mean_v[:, :3] - g.mean_v[:, :3]).astype(np.float64)
    assert abs(dm.std() - 0.01) < 5e-4 and abs(dm.mean()) < 5e-4
    v0, v1 = g.mean_v[:, 3].astype(np.float64), t.mean_v[:, 3].astype(np.float64)
    assert v1.min() >= 0.0 and v1.max() <= 1.0
    inside = (v1 > 0.0) & (v1 < 1.0)
    assert abs((v1 - v0)[inside].std() - 0.05) < 3e-3
    assert np.array_equal(t.logscale_w, g.logscale_w) and np.array_equal(t.quat, g.quat)
