"""VEG training oracle: opacity-guided maps, the image loss and the optimiser
step, stated plainly on the CPU in float64.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA library and never calls it.

What it computes (paper: Volume Encoding Gaussians, Sec. 4.2 "Training"):
  * opacity-guided training maps: the scalar range is divided into K steps;
    map k is centred in step k and falls off linearly with slope K;
  * the image loss (1 - lambda) L1 + lambda L_SSIM with lambda = 0.2, SSIM as
    defined by Wang et al. (2004);
  * the optimisation of the Gaussians' parameters, with the stored scalar and
    weight passed through a sigmoid (Sec. 3.3).

Readings where the paper is silent (each listed in the design notes):
  R13 map k: O_k(x) = max(0, 1 - s |x - c_k|), c_k = (k + 1/2)/K, slope s = K
      by default (a "broad" map halves it, a "narrow" map doubles it); the
      maps are tabulated like every TF (L entries at x = j/(L-1)).
  R17 SSIM per colour channel with an 11 x 11 Gaussian window of standard
      deviation 1.5 (normalised to sum 1), image borders padded with zeros
      (every output pixel has a full window), C1 = 0.01^2, C2 = 0.03^2 (the
      values of Wang et al. for a dynamic range of 1); the SSIM of a batch is
      the mean of the per-pixel, per-channel index over RGB; L_SSIM = 1 - SSIM.
      The transmittance channel takes part in neither loss.
  R18 optimiser: Adam (Kingma and Ba) per element with bias correction,
      beta1 = 0.9, beta2 = 0.999, eps = 1e-15; the scalar v and weight w are
      stored raw and activated by the logistic sigmoid; every other parameter
      (mean, log-scale, quaternion, normal, shininess, k_a, k_d, k_s) is used
      as stored.  Learning rates are per component (inputs).
"""
from __future__ import annotations

import numpy as np

SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2
SSIM_RADIUS = 5
SSIM_SIGMA = 1.5


# ----------------------------------------------------------------------------
# opacity-guided maps (Sec. 4.2, reading R13)
# ----------------------------------------------------------------------------

def tent_opacity(k, K, x, slope=None):
    """Opacity of map k of K at scalar values x."""
    s = float(K if slope is None else slope)
    c = (k + 0.5) / K
    return np.maximum(0.0, 1.0 - s * np.abs(np.asarray(x, np.float64) - c))


def tent_luts(K, rgb, slope=None):
    """K tables [K][L][4]: colour `rgb` (L, 3) shared by every map, opacity the
    tent of map k sampled at x_j = j/(L-1)."""
    rgb = np.asarray(rgb, np.float64)
    L = rgb.shape[0]
    x = np.arange(L) / (L - 1)
    out = np.zeros((K, L, 4))
    for k in range(K):
        out[k, :, :3] = rgb
        out[k, :, 3] = tent_opacity(k, K, x, slope)
    return out


# ----------------------------------------------------------------------------
# SSIM (Wang et al. 2004; reading R17)
# ----------------------------------------------------------------------------

def ssim_window():
    """The 11 x 11 window: outer product of a normalised 1-D Gaussian."""
    d = np.arange(-SSIM_RADIUS, SSIM_RADIUS + 1, dtype=np.float64)
    g = np.exp(-d * d / (2.0 * SSIM_SIGMA ** 2))
    g /= g.sum()
    return np.outer(g, g)


def _window_sum(img, win):
    """out[p] = sum_d win[d] img[p + d] over the window offsets d, zero
    outside the image (direct sum over every offset)."""
    H, W = img.shape
    r = SSIM_RADIUS
    pad = np.zeros((H + 2 * r, W + 2 * r))
    pad[r:r + H, r:r + W] = img
    out = np.zeros((H, W))
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            out += win[dy + r, dx + r] * pad[r + dy:r + dy + H, r + dx:r + dx + W]
    return out


def ssim_channel(x, y):
    """Per-pixel SSIM index of two single-channel images (H, W), and the
    partial derivatives of each pixel's index with respect to its local
    statistics mu_x, E[x^2] and E[xy] (for the gradient)."""
    win = ssim_window()
    mx, my = _window_sum(x, win), _window_sum(y, win)
    sxx, syy, sxy = _window_sum(x * x, win), _window_sum(y * y, win), _window_sum(x * y, win)
    vx, vy, cxy = sxx - mx * mx, syy - my * my, sxy - mx * my
    a1 = 2.0 * mx * my + SSIM_C1
    a2 = 2.0 * cxy + SSIM_C2
    b1 = mx * mx + my * my + SSIM_C1
    b2 = vx + vy + SSIM_C2
    s = a1 * a2 / (b1 * b2)
    # S = a1 a2 / (b1 b2) with a1, b1 functions of mu_x and a2, b2 functions
    # of mu_x, E[x^2], E[xy]:  d a1/d mu_x = 2 mu_y, d a2/d mu_x = -2 mu_y,
    # d b1/d mu_x = 2 mu_x, d b2/d mu_x = -2 mu_x, d b2/d E[x^2] = 1,
    # d a2/d E[xy] = 2.
    d_mx = (2.0 * my * a2 - 2.0 * my * a1) / (b1 * b2) - s * (2.0 * mx / b1 - 2.0 * mx / b2)
    d_sxx = -s / b2
    d_sxy = 2.0 * a1 / (b1 * b2)
    return s, d_mx, d_sxx, d_sxy


def ssim(out, target):
    """Mean SSIM over RGB of images [..., H, W, 4] and its gradient with
    respect to `out` (same shape, zero on the fourth channel)."""
    out = np.asarray(out, np.float64)
    target = np.asarray(target, np.float64)
    H, W = out.shape[-3], out.shape[-2]
    xs = out.reshape(-1, H, W, 4)
    ys = target.reshape(-1, H, W, 4)
    win = ssim_window()
    total = 0.0
    grad = np.zeros_like(xs)
    count = xs.shape[0] * H * W * 3
    for i in range(xs.shape[0]):
        for c in range(3):
            x, y = xs[i, :, :, c], ys[i, :, :, c]
            s, d_mx, d_sxx, d_sxy = ssim_channel(x, y)
            total += s.sum()
            # d S_q / d x_p = win[p - q] (d_mx_q + 2 x_p d_sxx_q + y_p d_sxy_q);
            # the window is symmetric, so the sum over q is a window sum.
            grad[i, :, :, c] = (_window_sum(d_mx, win) + 2.0 * x * _window_sum(d_sxx, win)
                                + y * _window_sum(d_sxy, win)) / count
    return total / count, grad.reshape(out.shape)


def l1_ssim_loss(out, target, lam=0.2):
    """(1 - lam) L1 + lam (1 - SSIM) over RGB and its gradient (Sec. 4.2).
    Returns (loss, l1, ssim, grad)."""
    out = np.asarray(out, np.float64)
    target = np.asarray(target, np.float64)
    d = out[..., :3] - target[..., :3]
    count = d.size
    l1 = np.abs(d).sum() / count
    s, gs = ssim(out, target)
    grad = np.zeros_like(out)
    grad[..., :3] = (1.0 - lam) * np.sign(d) / count
    grad -= lam * gs
    return (1.0 - lam) * l1 + lam * (1.0 - s), l1, s, grad


# ----------------------------------------------------------------------------
# optimiser (reading R18)
# ----------------------------------------------------------------------------

ADAM_BETA1 = 0.9
ADAM_BETA2 = 0.999
ADAM_EPS = 1e-15


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-np.asarray(x, np.float64)))


def activate(raw_mean_v, raw_logscale_w):
    """Rendered (mu, v) and (log-scale, w) from the stored raw arrays."""
    mv = np.array(raw_mean_v, np.float64)
    lw = np.array(raw_logscale_w, np.float64)
    mv[:, 3] = sigmoid(mv[:, 3])
    lw[:, 3] = sigmoid(lw[:, 3])
    return mv, lw


def adam_step(params, grads, m, v, lr, step):
    """One Adam step on the raw parameter arrays.

    params: list of five (N, 4) arrays (raw mean_v, raw logscale_w, quat,
    normal_beta, k_ads); grads: gradients with respect to the rendered
    (activated) values, same shapes; m, v: moment arrays (updated in place,
    like params); lr: (5, 4) learning rates per array and component; step:
    1-based iteration count.  The fourth component of arrays 0 and 1 is
    sigmoid-activated: its raw gradient is g s (1 - s), s = sigmoid(raw)."""
    bc1 = 1.0 - ADAM_BETA1 ** step
    bc2 = 1.0 - ADAM_BETA2 ** step
    for a in range(len(params)):
        g = np.array(grads[a], np.float64)
        if a < 2:
            s = sigmoid(params[a][:, 3])
            g[:, 3] = g[:, 3] * s * (1.0 - s)
        m[a][...] = ADAM_BETA1 * m[a] + (1.0 - ADAM_BETA1) * g
        v[a][...] = ADAM_BETA2 * v[a] + (1.0 - ADAM_BETA2) * g * g
        mhat = m[a] / bc1
        vhat = v[a] / bc2
        params[a][...] = params[a] - np.asarray(lr[a])[None, :] * mhat / (np.sqrt(vhat) + ADAM_EPS)
    return params
