"""Host-side parts of the training path (no GPU): the opacity-guided tables
and the raw-parameter store's activations, against the oracle."""
import numpy as np

from oracle import veg_train_oracle as TO
from paper_2504_13339_gb300 import scenes as S
from paper_2504_13339_gb300.train import _logit, default_lr, opacity_guided_luts


def test_opacity_guided_luts_match_oracle():
    rgb = S.colour_ramp(73)
    for K, slope in ((10, None), (5, 2.5), (20, 40.0), (1, None)):
        ours = opacity_guided_luts(K, rgb, slope)
        ref = TO.tent_luts(K, rgb, slope)
        assert ours.dtype == np.float32 and ours.shape == ref.shape
        assert np.abs(ours - ref).max() <= 1e-7


def test_logit_inverts_the_oracle_sigmoid():
    p = np.array([1e-3, 0.1, 0.5, 0.9, 0.999])
    assert np.allclose(TO.sigmoid(_logit(p)), p, rtol=1e-12)
    assert np.all(np.isfinite(_logit(np.array([0.0, 1.0]))))  # clamped


def test_default_learning_rates_follow_the_paper():
    lr = default_lr()
    assert lr.shape == (5, 4)
    assert lr[0, 3] == 2.5e-4 and lr[1, 3] == 2.5e-2  # scalar and weight (Sec. 5.1)
    assert lr[4, 3] == 0.0  # the unused fourth slot of (k_a, k_d, k_s, -)
    assert not default_lr(lighting=False)[3:].any()


def test_training_views_follow_the_orbit_grid():
    cams = S.grid_orbit_cameras(16, 10, 32, 32)
    assert len(cams) == 160
    eyes = np.stack([-c.world_to_cam[:, :3].T @ c.world_to_cam[:, 3] for c in cams])
    assert np.allclose(np.linalg.norm(eyes, axis=1), 3.0, atol=1e-5)


def test_field_gradient_matches_finite_differences():
    bf = S.blob_field(8, 3)
    p = np.random.default_rng(0).uniform(-1, 1, (7, 3))
    g = S.field_gradient(bf, p)
    h = 1e-6
    fd = np.stack([(bf.value(p + h * e) - bf.value(p - h * e)) / (2 * h) for e in np.eye(3)], 1)
    assert np.abs(g - fd).max() <= 1e-8 * max(1.0, np.abs(g).max())


def test_vertex_model_takes_vertices_and_their_values():
    vol = S.field_volume(S.blob_field(3, 5), 17)
    g, lt = S.vertex_model(vol, 300, 6)
    x = np.linspace(-1, 1, 17)
    idx = np.rint((g.mean_v[:, :3] + 1) * 8).astype(int)  # grid indices (x, y, z)
    assert np.allclose(x[idx], g.mean_v[:, :3], atol=1e-6)
    assert np.array_equal(g.mean_v[:, 3], vol[idx[:, 2], idx[:, 1], idx[:, 0]])
    assert len({tuple(r) for r in idx}) == 300  # without replacement
    assert lt.normal_beta.shape == (300, 4)


def test_pipeline_resize_keeps_buffers_while_the_count_fits():
    """After densification the pipeline adopts the new count in place while
    it fits the allocated rows (host logic; CPU tensors, no kernel runs)."""
    from paper_2504_13339_gb300 import build
    from paper_2504_13339_gb300.render import SplatPipeline
    build.build()
    cams = S.orbit_cameras(2, 125, 48, 32)
    p = SplatPipeline(100, cams, n_tf=1, device="cpu")
    p.ensure_shade_buffers()
    p.resize(110)  # beyond the rows: reallocated with headroom
    ptrs = [t.data_ptr() for t in p._rec], p.ws.data_ptr()
    for n in (120, 137, 60):
        p.resize(n)
        assert ([t.data_ptr() for t in p._rec], p.ws.data_ptr()) == ptrs
        assert p.geo.shape[0] == 2 * n and p.grad2d.shape[0] == 4 * n
        assert p.splat_shade.shape[0] == 2 * n and p.tiles.shape[0] == 2 * n
    p.resize(138)
    assert p.rows >= 138 and p.geo.shape[0] == 2 * 138 and p.splat_shade.shape[0] == 276
