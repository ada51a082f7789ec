"""Pins of the training oracle (no GPU): opacity-guided maps, SSIM and the
L1 + SSIM loss, Adam with the sigmoid activations.

Each check ties the oracle to something other than itself: closed forms,
library routines that compute the same quantity (scipy's Gaussian filter and
correlation, torch's Adam), invariants, and central finite differences.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi

from oracle import veg_oracle as O
from oracle import veg_train_oracle as TO

# Wang et al. (2004): C1 = (K1 L)^2, C2 = (K2 L)^2 with K1 = 0.01, K2 = 0.03 and
# dynamic range L = 1 for images in [0, 1]
C1 = (0.01 * 1.0) ** 2
C2 = (0.03 * 1.0) ** 2


# ----------------------------------------------------------------------------
# opacity-guided maps (Sec. 4.2, reading R13)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("K", [1, 5, 10, 20])
def test_tent_maps_partition_unity_and_shape(K):
    x = np.linspace(0.0, 1.0, 4001)
    total = sum(TO.tent_opacity(k, K, x) for k in range(K))
    inner = (x >= 0.5 / K) & (x <= 1.0 - 0.5 / K)
    assert np.allclose(total[inner], 1.0, atol=1e-12)  # every value equally weighted
    for k in range(K):
        c = (k + 0.5) / K
        assert TO.tent_opacity(k, K, c) == pytest.approx(1.0)
        assert TO.tent_opacity(k, K, c + 1.0 / K) == pytest.approx(0.0, abs=1e-12)
        # slope equal to the number of steps
        h = 0.1 / K
        assert (TO.tent_opacity(k, K, c) - TO.tent_opacity(k, K, c + h)) / h == pytest.approx(K)
    # broad / narrow maps: half and double slope
    assert TO.tent_opacity(0, K, 0.5 / K + 0.1 / K, slope=K / 2) == pytest.approx(0.95)
    assert TO.tent_opacity(0, K, 0.5 / K + 0.1 / K, slope=2 * K) == pytest.approx(0.8)


def test_tent_luts_tabulate_the_maps():
    rgb = np.random.default_rng(0).uniform(0, 1, (256, 3))
    luts = TO.tent_luts(10, rgb)
    assert luts.shape == (10, 256, 4)
    assert np.array_equal(luts[3, :, :3], rgb)
    j = np.arange(256)
    assert np.allclose(luts[3, :, 3], np.maximum(0, 1 - 10 * np.abs(j / 255 - 0.35)))


# ----------------------------------------------------------------------------
# SSIM (reading R17)
# ----------------------------------------------------------------------------

def test_window_is_the_normalised_gaussian_filter():
    """The window sum equals scipy's Gaussian filter (sigma 1.5, radius 5,
    zero padding) and scipy's correlation with the same window."""
    img = np.random.default_rng(1).uniform(0, 1, (23, 31))
    win = TO.ssim_window()
    assert win.shape == (11, 11) and win.sum() == pytest.approx(1.0)
    ours = TO._window_sum(img, win)
    gf = ndi.gaussian_filter(img, 1.5, truncate=5.0 / 1.5, mode="constant", cval=0.0)
    assert np.allclose(ours, gf, atol=1e-14)
    assert np.allclose(ours, ndi.correlate(img, win, mode="constant", cval=0.0), atol=1e-14)


def test_ssim_of_an_image_with_itself_is_one():
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, (2, 19, 21, 4))
    s, g = TO.ssim(x, x)
    assert s == pytest.approx(1.0, abs=1e-12)
    assert np.abs(g).max() < 1e-12


def test_ssim_constant_images_closed_form():
    """Constant images a, b: every full window has zero variance, so the
    index is (2ab + C1) / (a^2 + b^2 + C1) away from the zero-padded border."""
    a, b = 0.7, 0.3
    x = np.full((21, 24), a)
    y = np.full((21, 24), b)
    s = TO.ssim_channel(x, y)[0]
    ref = (2 * a * b + C1) / (a * a + b * b + C1)
    assert np.allclose(s[5:-5, 5:-5], ref, rtol=1e-12)
    assert not np.allclose(s[0, 0], ref)  # the border sees the zero padding


def test_ssim_linear_ramps_closed_form():
    """x = alpha i and y = beta i + gamma along the columns: under a full,
    symmetric window mu is the ramp itself and every (co)variance is
    (coefficients) x sigma_w^2 with sigma_w^2 = sum_d d^2 g(d) / sum_d g(d)
    of the 1-D window, so the index has a closed form that involves C2."""
    al, be, ga = 0.03, -0.02, 0.8
    H, W = 15, 30
    i = np.arange(W)[None, :].repeat(H, 0).astype(np.float64)
    x, y = al * i, be * i + ga
    d = np.arange(-5, 6)
    e = np.exp(-d * d / 4.5)
    var_w = float((d * d * e).sum() / e.sum())
    mx, my = al * i, be * i + ga
    ref = ((2 * mx * my + C1) * (2 * al * be * var_w + C2)
           / ((mx ** 2 + my ** 2 + C1) * ((al ** 2 + be ** 2) * var_w + C2)))
    s = TO.ssim_channel(x, y)[0]
    assert np.allclose(s[5:-5, 5:-5], ref[5:-5, 5:-5], rtol=1e-10)


def test_ssim_is_symmetric_and_bounded():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (17, 18))
    y = np.clip(x + rng.normal(0, 0.2, x.shape), 0, 1)
    sxy = TO.ssim_channel(x, y)[0]
    syx = TO.ssim_channel(y, x)[0]
    assert np.allclose(sxy, syx, atol=1e-14)
    assert np.all(sxy <= 1.0 + 1e-12) and np.all(sxy >= -1.0 - 1e-12)


def test_ssim_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, (2, 13, 17, 4))
    y = np.clip(x + rng.normal(0, 0.15, x.shape), 0, 1)
    _, g = TO.ssim(x, y)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (0, 6, 8, 1), (1, 12, 16, 2), (1, 3, 15, 0), (0, 12, 0, 2)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (TO.ssim(xp, y)[0] - TO.ssim(xm, y)[0]) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-6, abs=1e-10)
    assert np.all(g[..., 3] == 0)


def test_l1_ssim_loss_reduces_and_differentiates():
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, (1, 2, 12, 14, 4))
    y = rng.uniform(0, 1, x.shape)
    loss0, l1, s, g0 = TO.l1_ssim_loss(x, y, lam=0.0)
    ref, gref = O.l1_loss(x, y)  # pinned separately against its definition
    assert loss0 == pytest.approx(ref) and np.allclose(g0, gref)
    loss, l1b, sb, g = TO.l1_ssim_loss(x, y, lam=0.2)
    assert loss == pytest.approx(0.8 * l1b + 0.2 * (1 - sb))
    h = 1e-6
    for idx in [(0, 0, 3, 4, 0), (0, 1, 11, 13, 2), (0, 1, 0, 7, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (TO.l1_ssim_loss(xp, y)[0] - TO.l1_ssim_loss(xm, y)[0]) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-5, abs=1e-10)


# ----------------------------------------------------------------------------
# optimiser (reading R18)
# ----------------------------------------------------------------------------

def test_adam_matches_torch_adam_through_the_sigmoid():
    """Three steps of the oracle's Adam equal torch.optim.Adam (float64) on
    the raw parameters, the activated gradients chained by autograd."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    n = 37
    raw = [rng.normal(0, 1, (n, 4)) for _ in range(5)]
    lr = rng.uniform(1e-3, 1e-1, (5, 4))
    params = [r.copy() for r in raw]
    m = [np.zeros((n, 4)) for _ in range(5)]
    v = [np.zeros((n, 4)) for _ in range(5)]
    groups = []
    for a in range(5):
        for c in range(4):
            groups.append({"params": [], "lr": float(lr[a, c])})
    # one tensor per (array, component) so each can have its own rate
    cols = [[torch.tensor(raw[a][:, c], dtype=torch.float64, requires_grad=True)
             for c in range(4)] for a in range(5)]
    for a in range(5):
        for c in range(4):
            groups[a * 4 + c]["params"].append(cols[a][c])
    opt = torch.optim.Adam(groups, betas=(TO.ADAM_BETA1, TO.ADAM_BETA2), eps=TO.ADAM_EPS)
    for step in range(1, 4):
        g_act = [rng.normal(0, 1, (n, 4)) for _ in range(5)]
        TO.adam_step(params, g_act, m, v, lr, step)
        opt.zero_grad()
        loss = 0
        for a in range(5):
            for c in range(4):
                x = cols[a][c]
                act = torch.sigmoid(x) if (a < 2 and c == 3) else x
                loss = loss + (torch.tensor(g_act[a][:, c]) * act).sum()
        loss.backward()
        opt.step()
    for a in range(5):
        for c in range(4):
            assert np.allclose(params[a][:, c], cols[a][c].detach().numpy(), rtol=1e-12,
                               atol=1e-14)


def test_adam_first_step_closed_form_and_zero_gradient():
    n = 5
    p = [np.zeros((n, 4)) for _ in range(5)]
    m = [np.zeros((n, 4)) for _ in range(5)]
    v = [np.zeros((n, 4)) for _ in range(5)]
    g = [np.zeros((n, 4)) for _ in range(5)]
    g[2][:, 1] = np.array([3.0, -2.0, 0.5, -1e-3, 0.0])
    lr = np.full((5, 4), 0.01)
    TO.adam_step(p, g, m, v, lr, 1)
    # m_hat = g, v_hat = g^2: the first step moves by lr sign(g)
    assert np.allclose(p[2][:, 1], -0.01 * np.sign(g[2][:, 1]), atol=1e-12)
    for a in (0, 1, 3, 4):
        assert not p[a].any()
    # the sigmoid chain: raw gradient of the activated 4th component
    s = TO.sigmoid(0.0)
    p2 = [np.zeros((n, 4)) for _ in range(5)]
    g2 = [np.zeros((n, 4)) for _ in range(5)]
    g2[0][:, 3] = 4.0
    m2 = [np.zeros((n, 4)) for _ in range(5)]
    v2 = [np.zeros((n, 4)) for _ in range(5)]
    TO.adam_step(p2, g2, m2, v2, lr, 1)
    assert np.allclose(m2[0][:, 3], 0.1 * 4.0 * s * (1 - s))
    mv, lw = TO.activate(p2[0], p2[1])
    assert np.allclose(mv[:, 3], TO.sigmoid(p2[0][:, 3])) and np.allclose(lw[:, 3], 0.5)
