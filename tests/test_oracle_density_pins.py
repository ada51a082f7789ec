"""Pins of the adaptive-density-control oracle (no GPU).

Brute-force recomputation of the statistic on small inputs, hand-built cases
for every decision and its boundary, closed forms for the thresholds and the
split scale, and a statistical check of the split sampling against the
covariance built from Hamilton products (independent of the oracle's
rotation matrix).
"""
import math

import numpy as np
import pytest

from oracle import veg_density_oracle as D


def test_statistic_brute_force():
    rng = np.random.default_rng(0)
    V, N, W, H = 3, 50, 120, 80
    g = rng.normal(0, 1e-3, (V, N, 2)).astype(np.float32)
    tiles = rng.integers(0, 3, (V, N)).astype(np.int32)
    acc = np.zeros(N, np.float32)
    cnt = np.zeros(N, np.int32)
    for _ in range(2):  # two iterations
        D.grad_stat_update(acc, cnt, g, tiles, W, H)
    for i in range(N):
        ref_sum, ref_cnt = 0.0, 0
        for v in range(V):
            if tiles[v, i] > 0:
                ref_sum += 2 * math.hypot(g[v, i, 0] * W / 2, g[v, i, 1] * H / 2)
                ref_cnt += 2
        assert cnt[i] == ref_cnt
        assert acc[i] == pytest.approx(ref_sum, rel=1e-6, abs=1e-12)


def test_thresholds_closed_forms():
    th = D.thresholds(3.3)
    w = 1.0 / (1.0 + math.exp(-float(th["raw_weight"])))
    assert w == pytest.approx(0.005, rel=1e-6)
    assert math.exp(float(th["log_size"])) == pytest.approx(0.033, rel=1e-6)
    assert math.exp(float(th["log_split"])) == pytest.approx(1.6, rel=1e-7)
    assert float(th["grad"]) == pytest.approx(2e-4, rel=1e-7)


def test_scene_extent_of_an_orbit():
    az = np.linspace(0, 2 * np.pi, 16, endpoint=False)
    c = np.stack([3 * np.sin(az), np.zeros(16), 3 * np.cos(az)], 1)
    assert D.scene_extent(c) == pytest.approx(3.3)
    # distances are taken from the cameras' centroid, not from the origin
    shifted = c + np.array([10.0, -4.0, 2.0])
    assert D.scene_extent(shifted) == pytest.approx(3.3)
    assert D.scene_extent([[10.0, 0, 0], [12.0, 0, 0]]) == pytest.approx(1.1)


def _model(n, rng, ls=-4.0):
    mv = np.concatenate([rng.normal(0, 0.3, (n, 3)), rng.normal(0, 1, (n, 1))], 1)
    lw = np.concatenate([np.full((n, 3), ls) + rng.normal(0, 0.1, (n, 3)),
                         rng.normal(0, 1, (n, 1))], 1)
    q = rng.standard_normal((n, 4))
    return [mv.astype(np.float32), lw.astype(np.float32), q.astype(np.float32),
            rng.normal(0, 1, (n, 4)).astype(np.float32), rng.uniform(0, 1, (n, 4)).astype(np.float32)]


def test_classification_and_boundaries():
    th = D.thresholds(3.3)
    n = 8
    p = _model(n, np.random.default_rng(1))
    lw = p[1]
    lw[:, 3] = 2.0  # well above the prune threshold
    acc = np.zeros(n, np.float32)
    cnt = np.ones(n, np.int32)
    acc[0] = th["grad"]                  # average exactly at the threshold: densified
    lw[0, :3] = th["log_size"]           # size exactly at the threshold: cloned (strict >)
    acc[1] = th["grad"] * 2
    lw[1, 0] = th["log_size"] + np.float32(1e-3)  # one axis above: split
    acc[2] = np.nextafter(th["grad"], np.float32(0))  # just below: kept
    acc[3] = th["grad"] * 10
    lw[3, 3] = th["raw_weight"]          # weight exactly at the threshold: not pruned
    acc[4] = th["grad"] * 10
    lw[4, 3] = np.nextafter(th["raw_weight"], np.float32(-10))  # just below: pruned
    cnt[5] = 0                           # never seen: kept
    acc[5] = 1.0
    acc[6] = th["grad"] * 4
    cnt[6] = 4                           # average exactly at the threshold again
    lw[6, :3] = -10.0
    acc[7] = th["grad"] * 3
    cnt[7] = 4                           # average below
    act = D.classify(lw, acc, cnt, th)
    assert list(act) == [D.CLONE, D.SPLIT, D.KEEP, D.CLONE, D.PRUNE, D.KEEP, D.CLONE, D.KEEP]


def test_outputs_order_copies_and_moments():
    th = D.thresholds(3.3)
    rng = np.random.default_rng(2)
    n = 6
    p = _model(n, rng)
    p[1][:, 3] = 1.0
    m = [rng.normal(0, 1, (n, 4)) for _ in range(5)]
    v = [rng.uniform(0, 1, (n, 4)) for _ in range(5)]
    acc = np.array([0, 1, 1, 0, 1, 0], np.float32)
    cnt = np.ones(n, np.int32)
    p[1][2, :3] = 0.0         # big: split
    p[1][3, 3] = -8.0         # pruned
    z = rng.standard_normal((n, 2, 3))
    out, om, ov, act = D.densify(p, m, v, acc, cnt, z, th)
    assert list(act) == [D.KEEP, D.CLONE, D.SPLIT, D.PRUNE, D.CLONE, D.KEEP]
    # keep, clone pair, two children, (pruned), clone pair, keep
    src = [0, 1, 1, 2, 2, 4, 4, 5]
    assert out[0].shape == (8, 4)
    fresh = {2, 3, 4, 6}
    for k, i in enumerate(src):
        for a in range(5):
            if k in (3, 4) and a in (0, 1):
                continue  # split children differ in mean and scale
            assert np.array_equal(out[a][k], p[a][i].astype(np.float64))
            assert np.array_equal(om[a][k], 0 * m[a][i] if k in fresh else m[a][i])
            assert np.array_equal(ov[a][k], 0 * v[a][i] if k in fresh else v[a][i])
    for k, j in ((3, 0), (4, 1)):
        assert np.allclose(np.exp(out[1][k, :3]) * 1.6, np.exp(p[1][2, :3].astype(np.float64)),
                           rtol=1e-6)
        assert out[1][k, 3] == p[1][2, 3]


def _rotate(q, v):
    """v rotated by the unit quaternion q = (w, x, y, z): q v q*."""
    w, x, y, z = q

    def mul(a, b):
        return np.array([a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3],
                         a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2],
                         a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1],
                         a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0]])
    return mul(mul(q, np.array([0.0, *v])), np.array([w, -x, -y, -z]))[1:]


def test_split_children_sample_the_gaussian():
    """Children of one Gaussian, over many draws, have its mean and
    covariance R diag(s^2) R^T (R from Hamilton products)."""
    th = D.thresholds(3.3)
    rng = np.random.default_rng(3)
    n = 20000
    q = np.array([0.8, -0.3, 0.4, 0.2])
    q /= np.linalg.norm(q)
    ls = np.array([-1.0, -2.0, -1.5])
    mu = np.array([0.1, -0.2, 0.3])
    p = [np.tile(np.r_[mu, 0.0], (n, 1)).astype(np.float32),
         np.tile(np.r_[ls, 2.0], (n, 1)).astype(np.float32),
         np.tile(q, (n, 1)).astype(np.float32), None, None]
    zeros = [None if a is None else np.zeros_like(a) for a in p]
    acc = np.ones(n, np.float32)
    cnt = np.ones(n, np.int32)
    z = rng.standard_normal((n, 2, 3))
    out, _, _, act = D.densify(p, zeros, zeros, acc, cnt, z, th)
    assert np.all(act == D.SPLIT) and out[0].shape[0] == 2 * n
    x = out[0][:, :3]
    R = np.stack([_rotate(q, e) for e in np.eye(3)], 1)
    s = np.exp(ls)
    cov = R @ np.diag(s * s) @ R.T
    assert np.allclose(x.mean(0), mu, atol=4 * s.max() / np.sqrt(2 * n))
    assert np.allclose(np.cov(x.T), cov, atol=0.03 * np.abs(cov).max())
