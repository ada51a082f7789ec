"""Blinn-Phong shading (Eq. 2-3) on the GPU vs the CPU oracle, through the C ABI.

Bars: shading factors within a bound derived from float32 rounding (the
specular power amplifies the error of n.h by at most beta); shaded images
within 1e-4 max-abs and n_contrib equal on every pixel (threshold-straddling
pixels matched to the oracle's outcome with the same decisions, as for
unshaded renders, see tests/parity.py); gradients within a relative 1e-3 of
the oracle's largest entry per tensor and, per element, 1e-3 |g_ref| + 1e-6
max |g_ref|.
"""
import numpy as np
import pytest
import torch

from oracle import veg_oracle as O
from paper_2504_13339_gb300 import scenes as S
from paper_2504_13339_gb300.render import SplatPipeline, headlight_dirs, lut_tensor, render
from parity import checked_forward, grad_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def lit_scene(n=2000):
    g = S.uniform_gaussians(2000, 31, logscale_mean=-3.0, logscale_std=0.4)
    g.logscale_w[:, 3] = np.random.default_rng(32).uniform(0.3, 1.0, g.n)
    g = g.subset(np.arange(n))
    cams = S.orbit_cameras(3, 33, 100, 70)  # ragged 7 x 5 tiles
    lt = S.random_lighting(g.n, 50)
    return g, cams, lt


def lights_of(cams, kind):
    if kind == "headlight":
        return np.stack([O.headlight(c) for c in cams])
    d = np.array([[0.3, 0.8, 0.5], [-0.6, 0.2, 0.77], [0.0, -1.0, 0.1]])
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def lit_forward(g, cams, tfs, lt, lights, bg=(0.0, 0.0, 0.0)):
    p = SplatPipeline(g.n, cams, n_tf=len(tfs))
    tens = (dev(g.mean_v), dev(g.logscale_w), dev(g.quat))
    lit = (dev(lt.normal_beta), dev(lt.k_ads))
    luts = lut_tensor(tfs)
    p.project(*tens, luts)
    p.shade(tens[0], *lit, lights)
    p.bin_sort()
    p.composite(luts, bg)
    torch.cuda.synchronize()
    return p, tens, lit, luts


def check(name, out, nc, fwd, proj, cams, bins, tfs, bg=(0.0, 0.0, 0.0), region=None):
    """Image parity against the oracle's forward; returns the mask of pixels
    whose upstream gradient is zeroed."""
    return checked_forward(name, fwd, proj, cams, bins, tfs, bg, out, nc, region)


def test_headlight_directions_agree_with_oracle():
    cams = S.orbit_cameras(5, 60, 64, 64)
    assert np.allclose(headlight_dirs(cams), lights_of(cams, "headlight"), atol=1e-12)


@pytest.mark.parametrize("kind", ["headlight", "fixed"])
def test_shade_factors_match_oracle(kind):
    g, cams, lt = lit_scene()
    lights = lights_of(cams, kind)
    p = SplatPipeline(g.n, cams, n_tf=1)
    p.shade(dev(g.mean_v), dev(lt.normal_beta), dev(lt.k_ads), lights)
    torch.cuda.synchronize()
    got = p.splat_shade.cpu().numpy().reshape(len(cams), g.n, 2)
    d = lt.as_dict(lights)
    for v, cam in enumerate(cams):
        f = O.shade64(cam, lights[v], g.mean_v[:, :3].astype(np.float64), d["normal"], d["ka"],
                      d["kd"], d["ks"], d["beta"])
        assert np.all(np.abs(got[v, :, 0] - f["s_d"]) <= 2e-6 * (1 + np.abs(f["s_d"])))
        # float32 error of n.h (a few 1e-7) times the power's slope <= beta k_s
        tol = 1e-6 + 4e-6 * d["beta"] * d["ks"]
        assert np.all(np.abs(got[v, :, 1] - f["s_s"]) <= tol)


@pytest.mark.parametrize("kind", ["headlight", "fixed"])
def test_lit_render_matches_oracle(kind):
    g, cams, lt = lit_scene()
    tfs = S.bump_tfs(2, 51)
    bg = (0.1, 0.2, 0.0)
    lights = lights_of(cams, kind)
    p, *_ = lit_forward(g, cams, tfs, lt, lights, bg)
    proj, bins, fwd = O.render(cams, g, tfs, bg=bg, lighting=lt.as_dict(lights))
    check(f"lit_{kind}", p.out.cpu().numpy(), p.n_contrib.cpu().numpy(), fwd, proj, cams, bins,
          tfs, bg)


def test_trivial_material_equals_unshaded_render():
    """k_a = 1, k_d = k_s = 0 gives s_d = 1, s_s = 0: the shaded forward is
    bit-identical to the unshaded one and the backward agrees to rounding."""
    g, cams, lt = lit_scene(900)
    lt.k_ads[:] = np.array([1.0, 0.0, 0.0, 0.0], np.float32)
    tfs = S.bump_tfs(3, 52)
    lights = lights_of(cams, "headlight")
    p, tens, lit, luts = lit_forward(g, cams, tfs, lt, lights)
    q = SplatPipeline(g.n, cams, n_tf=len(tfs))
    q.project(*tens, luts)
    q.bin_sort()
    q.composite(luts)
    torch.cuda.synchronize()
    assert torch.equal(p.out, q.out) and torch.equal(p.n_contrib, q.n_contrib)
    dout = dev(np.random.default_rng(53).standard_normal(p.out.shape).astype(np.float32))
    ga = [torch.zeros_like(t) for t in tens]
    gb = [torch.zeros_like(t) for t in tens]
    gn, gk = torch.zeros_like(lit[0]), torch.zeros_like(lit[1])
    p.backward(dout, *ga, gn, gk)
    q.backward(dout, *gb)
    torch.cuda.synchronize()
    for a, b in zip(ga, gb):
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-5 * float(b.abs().max()))
    assert float(p.grad_shade[:, 1].abs().max()) > 0  # ds_s is live even with k_s = 0


@pytest.mark.parametrize("kind", ["headlight", "fixed"])
def test_lit_backward_matches_oracle(kind):
    g, cams, lt = lit_scene(700)
    tfs = S.bump_tfs(2, 54)
    bg = (0.1, 0.0, 0.2)
    lights = lights_of(cams, kind)
    p, tens, lit, luts = lit_forward(g, cams, tfs, lt, lights, bg)
    d = lt.as_dict(lights)
    proj, bins, fwd = O.render(cams, g, tfs, bg=bg, record=True, lighting=d)
    excl = check(f"lit_backward_{kind}", p.out.cpu().numpy(), p.n_contrib.cpu().numpy(), fwd,
                 proj, cams, bins, tfs, bg)
    dout = np.random.default_rng(55).standard_normal(fwd["out"].shape)
    dout[excl] = 0.0
    grads = [torch.zeros_like(t) for t in tens]
    gn, gk = torch.zeros_like(lit[0]), torch.zeros_like(lit[1])
    p.backward(dev(dout.astype(np.float32)), *grads, gn, gk)
    torch.cuda.synchronize()
    g2 = O.composite_bwd(proj, cams, bins, tfs, bg, fwd, dout)
    got2 = p.grad2d.cpu().numpy().reshape(len(cams), g.n, 8)
    gsh = p.grad_shade.cpu().numpy().reshape(len(cams), g.n, 2)
    for k, name in enumerate(["du_x", "du_y", "da", "db", "dc", "dv", "dw"]):
        grad_check(got2[..., k], g2[..., k], name)
    grad_check(gsh[..., 0], g2[..., 7], "ds_d")
    grad_check(gsh[..., 1], g2[..., 8], "ds_s")
    gm, gl, gq = O.params_grad(cams, g, proj, g2)
    dn, dka, dkd, dks, db, dm_sh = O.lighting_grad(cams, g, d, proj, g2)
    grad_check(grads[0].cpu().numpy()[:, :3], gm[:, :3] + dm_sh, "mean")
    grad_check(grads[0].cpu().numpy()[:, 3], gm[:, 3], "v")
    grad_check(grads[1].cpu().numpy()[:, :3], gl[:, :3], "logscale")
    grad_check(grads[1].cpu().numpy()[:, 3], gl[:, 3], "w")
    grad_check(grads[2].cpu().numpy(), gq, "quat")
    gn, gk = gn.cpu().numpy(), gk.cpu().numpy()
    grad_check(gn[:, :3], dn, "normal")
    grad_check(gn[:, 3], db, "beta")
    grad_check(gk[:, 0], dka, "k_a")
    grad_check(gk[:, 1], dkd, "k_d")
    grad_check(gk[:, 2], dks, "k_s")
    assert not gk[:, 3].any()


def test_lit_autograd_function():
    g, cams, lt = lit_scene(1200)
    tfs = S.bump_tfs(1, 56)
    luts = lut_tensor(tfs)
    lights = headlight_dirs(cams)
    p = SplatPipeline(g.n, cams, n_tf=1)
    mean_v = dev(g.mean_v).requires_grad_()
    ls, q = dev(g.logscale_w).requires_grad_(), dev(g.quat).requires_grad_()
    nb, k = dev(lt.normal_beta).requires_grad_(), dev(lt.k_ads).requires_grad_()
    out = render(mean_v, ls, q, p, luts, (0.0, 0.0, 0.0), normal_beta=nb, k_ads=k,
                 light_dirs=lights)
    w = torch.randn_like(out)
    (out * w).sum().backward()
    ref = [torch.zeros_like(t) for t in (mean_v, ls, q, nb, k)]
    p.backward(w.contiguous(), *ref)
    close = lambda x, y: bool(((x - y).abs() <= 1e-5 * y.abs().max() + 1e-4 * y.abs()).all())
    for got, r in zip((mean_v.grad, ls.grad, q.grad, nb.grad, k.grad), ref):
        assert close(got, r)


def test_lit_one_table_per_view_matches_oracle():
    """Shading with one table per view (veg_tf.view_tf): the TG = 1 shaded
    forward and backward against the oracle rendering each view with its
    own table."""
    from paper_2504_13339_gb300 import _lib
    g, cams, lt = lit_scene(700)
    tfs = S.bump_tfs(3, 57)
    view_tf = [2, 0, 1]
    lights = lights_of(cams, "headlight")
    p = SplatPipeline(g.n, cams, n_tf=1)
    tens = (dev(g.mean_v), dev(g.logscale_w), dev(g.quat))
    lit = (dev(lt.normal_beta), dev(lt.k_ads))
    luts = lut_tensor(tfs)
    vt = torch.as_tensor(np.asarray(view_tf, np.int32), device="cuda")
    desc = _lib.tf_desc(luts, vt)
    p.project(*tens, None)
    p.shade(tens[0], *lit, lights)
    p.bin_sort()
    _lib.veg_composite_fwd(p.c_cams, p.n, p.geo, p.aux, p.vals, p.ranges, desc, (0, 0, 0), 0,
                           p.out, p.n_contrib, tile_order=p.order, splat_shade=p.splat_shade)
    dout = np.random.default_rng(58).standard_normal(p.out.shape)
    d = lt.as_dict(lights)
    refs = []
    for v, cam in enumerate(cams):
        dv_ = {**d, "lights": d["lights"][v:v + 1]}
        tv = tfs[view_tf[v]:view_tf[v] + 1]
        proj, bins, fwd = O.render([cam], g, tv, cull=False, record=True, lighting=dv_)
        excl = check(f"lit_view_tf_{v}", p.out.cpu().numpy()[v:v + 1],
                     p.n_contrib.cpu().numpy()[v:v + 1], fwd, proj, [cam], bins, tv)
        dd = dout[v:v + 1].copy()
        dd[excl] = 0.0
        dout[v:v + 1] = dd
        refs.append((proj, bins, fwd, dv_, cam))
    grads = [torch.zeros_like(t) for t in tens]
    gn, gk = torch.zeros_like(lit[0]), torch.zeros_like(lit[1])
    _lib.veg_composite_bwd(p.c_cams, p._g, p.geo, p.aux, p.tiles,
                           p.vals, p.ranges, desc, (0, 0, 0), 0, p.out, p.n_contrib,
                           dev(dout.astype(np.float32)), None, grads[0], grads[1], grads[2],
                           p.grad2d, tile_order=p.order, splat_shade=p.splat_shade,
                           grad_shade=p.grad_shade)
    _lib.veg_shade_bwd(p.c_cams, tens[0], lit[0], lit[1], lights, p.tiles, p.grad_shade,
                       grads[0], gn, gk)
    torch.cuda.synchronize()
    gm = np.zeros((g.n, 4))
    gl = np.zeros((g.n, 4))
    gq = np.zeros((g.n, 4))
    gnr = np.zeros((g.n, 4))
    gkr = np.zeros((g.n, 4))
    for v, (proj, bins, fwd, dv_, cam) in enumerate(refs):
        t = tfs[view_tf[v]:view_tf[v] + 1]
        g2 = O.composite_bwd(proj, [cam], bins, t, (0, 0, 0), fwd, dout[v:v + 1])
        a, b, c = O.params_grad([cam], g, proj, g2)
        dn, dka, dkd, dks, db, dm = O.lighting_grad([cam], g, dv_, proj, g2)
        gm += a
        gm[:, :3] += dm
        gl += b
        gq += c
        gnr[:, :3] += dn
        gnr[:, 3] += db
        gkr[:, 0] += dka
        gkr[:, 1] += dkd
        gkr[:, 2] += dks
    grad_check(grads[0].cpu().numpy(), gm, "mean_v")
    grad_check(grads[1].cpu().numpy(), gl, "logscale_w")
    grad_check(grads[2].cpu().numpy(), gq, "quat")
    grad_check(gn.cpu().numpy(), gnr, "normal_beta")
    grad_check(gk.cpu().numpy(), gkr, "k_ads")


def test_full_size_lit_crop_gradients():
    """The shaded training step's scene at full size (1M Gaussians, 1024^2,
    4 TFs, headlight): every gradient of a loss on a 64x64 crop against the
    oracle, for the Gaussians the crop touches; all others stay zero."""
    g, _, cams, tfs = S.train_scene()
    cam = cams[0]
    lt = S.random_lighting(g.n, 3)
    lights = np.stack([O.headlight(cam)])
    p = SplatPipeline(g.n, cams, n_tf=len(tfs), capacity=16_000_000)
    tens = (dev(g.mean_v), dev(g.logscale_w), dev(g.quat))
    lit = (dev(lt.normal_beta), dev(lt.k_ads))
    luts = lut_tensor(tfs)
    p.project(*tens, luts)
    p.shade(tens[0], *lit, lights)
    p.bin_sort()
    p.composite(luts)
    x0 = y0 = 480
    tiles = [(y0 // 16 + j) * cam.tiles_x + x0 // 16 + i for j in range(4) for i in range(4)]
    d = lt.as_dict(lights)
    pr = O.project32(cam, g, tfs)
    O.attach_shading([pr], [cam], g, d)
    bins = O.bins_from_lists([O.tile_lists(pr, cam, tiles)], 1, cam.tiles_x * cam.tiles_y)
    fwd = O.composite_fwd([pr], cams, bins, tfs, tiles=tiles, record=True)
    region = np.zeros(fwd["flag"].shape, bool)
    region[..., y0:y0 + 64, x0:x0 + 64] = True
    excl = check("lit_train_1M_crop", p.out.cpu().numpy(), p.n_contrib.cpu().numpy(), fwd, [pr],
                 cams, bins, tfs, region=region)
    dout = np.zeros(fwd["out"].shape)
    dout[..., y0:y0 + 64, x0:x0 + 64, :] = np.random.default_rng(57).standard_normal(
        (1, len(tfs), 64, 64, 4))
    dout[excl] = 0.0
    grads = [torch.zeros_like(t) for t in tens]
    gn, gk = torch.zeros_like(lit[0]), torch.zeros_like(lit[1])
    p.backward(dev(dout.astype(np.float32)), *grads, gn, gk)
    torch.cuda.synchronize()
    g2 = O.composite_bwd([pr], cams, bins, tfs, (0, 0, 0), fwd, dout, tiles=tiles)
    touched = np.nonzero(np.abs(g2[0]).sum(1))[0]
    assert touched.size > 100
    gs = g.subset(touched)
    prs = {k: (v[touched] if isinstance(v, np.ndarray) and v.shape[:1] == (g.n,) else v)
           for k, v in pr.items()}
    ds = {k: (v[touched] if k != "lights" else v) for k, v in d.items()}
    gm, gl, gq = O.params_grad(cams, gs, [prs], g2[:, touched])
    dn, dka, dkd, dks, db, dm_sh = O.lighting_grad(cams, gs, ds, [prs], g2[:, touched])
    got = [t.cpu().numpy() for t in grads]
    gn, gk = gn.cpu().numpy(), gk.cpu().numpy()
    others = np.setdiff1d(np.arange(g.n), touched)
    for a in got + [gn, gk]:
        assert not a[others].any()
    grad_check(got[0][touched, :3], gm[:, :3] + dm_sh, "mean")
    grad_check(got[0][touched, 3], gm[:, 3], "v")
    grad_check(got[1][touched, :3], gl[:, :3], "logscale")
    grad_check(got[1][touched, 3], gl[:, 3], "w")
    grad_check(got[2][touched], gq, "quat")
    grad_check(gn[touched, :3], dn, "normal")
    grad_check(gn[touched, 3], db, "beta")
    grad_check(gk[touched, 0], dka, "k_a")
    grad_check(gk[touched, 1], dkd, "k_d")
    grad_check(gk[touched, 2], dks, "k_s")
