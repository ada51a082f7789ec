"""Training path on the GPU vs the CPU oracle (Sec. 4.2): the L1 + SSIM loss
and its gradient, the Adam step, one opacity-guided training iteration, and
a short training run.

Bars: loss values within a relative 1e-5; loss gradients within 1e-3 of the
oracle's largest entry (measured far below); Adam displacements within a
relative 1e-4 of the largest displacement per array; the gradients of a
training iteration within 1e-3 of the oracle's largest entry per tensor.
"""
import numpy as np
import pytest
import torch

from oracle import veg_oracle as O
from oracle import veg_train_oracle as TO
from paper_2504_13339_gb300 import _lib, scenes as S
from paper_2504_13339_gb300.render import lut_tensor
from paper_2504_13339_gb300.train import OpacityGuidedTrainer, TrainParams, opacity_guided_luts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")


def gpu_loss(out, tgt, lam=0.2):
    H, W = out.shape[-3], out.shape[-2]
    n_img = out.size // (H * W * 4)
    o, t = dev(out), dev(tgt)
    grad = torch.empty_like(o)
    loss = torch.zeros(3, device="cuda")
    ws = torch.empty(_lib.veg_l1_ssim_loss_workspace_size(n_img, H, W), dtype=torch.uint8,
                     device="cuda")
    _lib.veg_l1_ssim_loss(o, t, grad, loss, ws, lam)
    torch.cuda.synchronize()
    return loss.cpu().numpy().astype(np.float64), grad.cpu().numpy()


def image_pair(shape, seed, noise=0.1):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, shape).astype(np.float32)
    # smooth structure plus noise, as rendered images have
    x[..., :3] = (0.5 + 0.4 * np.sin(np.linspace(0, 6, shape[-2]))[None, :, None]
                  * np.cos(np.linspace(0, 4, shape[-3]))[:, None, None] + 0.1 * x[..., :3])
    y = np.clip(x + rng.normal(0, noise, shape), 0, 1).astype(np.float32)
    return x, y


@pytest.mark.parametrize("shape,lam", [((2, 37, 29, 4), 0.2), ((1, 48, 64, 4), 0.2),
                                       ((3, 16, 16, 4), 1.0), ((1, 21, 50, 4), 0.0)])
def test_l1_ssim_loss_matches_oracle(shape, lam):
    x, y = image_pair(shape, 60 + shape[1])
    (loss, l1, ss), g = gpu_loss(x, y, lam)
    ref, rl1, rss, gref = TO.l1_ssim_loss(x, y, lam)
    assert loss == pytest.approx(ref, rel=1e-5, abs=1e-7)
    assert l1 == pytest.approx(rl1, rel=1e-5) and ss == pytest.approx(rss, rel=1e-5)
    err = np.abs(g - gref).max() / np.abs(gref).max()
    assert err <= 1e-3, err
    assert not g[..., 3].any()


def test_l1_ssim_of_identical_images():
    x, _ = image_pair((2, 40, 33, 4), 70)
    (loss, l1, ss), g = gpu_loss(x, x)
    assert l1 == 0.0 and ss == pytest.approx(1.0, abs=1e-6) and loss == pytest.approx(0, abs=1e-6)
    # the L1 part is exactly zero (sign 0) and the SSIM part vanishes up to
    # rounding: per element at most 1e-3 / count (an L1 gradient is 0.8 / count)
    assert np.abs(g).max() * (2 * 40 * 33 * 3) <= 1e-3


def test_l1_ssim_full_size_on_a_crop():
    """4 images of 1024 x 1024 (the training-step size): the loss in full and
    the gradient on a 64 x 64 crop, whose exact value the oracle gets from
    the crop plus a 10-pixel margin (the gradient at a pixel depends only on
    pixels within 10 of it)."""
    x, y = image_pair((4, 1024, 1024, 4), 71, noise=0.05)
    (loss, l1, ss), g = gpu_loss(x, y)
    rl1 = np.abs(x[..., :3].astype(np.float64) - y[..., :3]).mean()
    assert l1 == pytest.approx(rl1, rel=1e-5)
    i, y0, x0 = 2, 500, 300
    cx = x[i:i + 1, y0 - 10:y0 + 74, x0 - 10:x0 + 74]
    cy = y[i:i + 1, y0 - 10:y0 + 74, x0 - 10:x0 + 74]
    _, _, _, gref = TO.l1_ssim_loss(cx, cy)
    count_full, count_crop = 4 * 1024 * 1024 * 3, 84 * 84 * 3
    got = g[i, y0:y0 + 64, x0:x0 + 64] * count_full
    ref = gref[0, 10:74, 10:74] * count_crop
    assert np.abs(got - ref).max() <= 1e-3 * np.abs(ref).max()
    # SSIM of one full image via the oracle's statistics
    s = np.mean([TO.ssim_channel(x[0, :, :, c].astype(np.float64),
                                 y[0, :, :, c].astype(np.float64))[0].mean() for c in range(3)])
    (_, _, ss0), _ = gpu_loss(x[:1], y[:1])
    assert ss0 == pytest.approx(s, rel=1e-5)


def test_adam_matches_oracle():
    rng = np.random.default_rng(72)
    n = 3001
    raw = [rng.normal(0, 1, (n, 4)).astype(np.float32) for _ in range(5)]
    lr = rng.uniform(1e-3, 5e-2, (5, 4))
    p = [dev(r) for r in raw]
    gr = [torch.zeros_like(t) for t in p]
    m = [torch.zeros_like(t) for t in p]
    v = [torch.zeros_like(t) for t in p]
    rend = [torch.zeros_like(p[0]), torch.zeros_like(p[1])]
    arrays = _lib.adam_arrays(p, gr, m, v, rend)
    ref = [r.astype(np.float64) for r in raw]
    rm = [np.zeros((n, 4)) for _ in range(5)]
    rv = [np.zeros((n, 4)) for _ in range(5)]
    for step in range(1, 5):
        g = [rng.normal(0, 1, (n, 4)).astype(np.float32) for _ in range(5)]
        g[1][::7] = 0.0  # zero gradients leave the values unchanged at step 1
        for a in range(5):
            gr[a].copy_(dev(g[a]))
        _lib.veg_adam_step(arrays, n, lr, step)
        TO.adam_step(ref, g, rm, rv, lr, step)
    torch.cuda.synchronize()
    for a in range(5):
        got = p[a].cpu().numpy().astype(np.float64) - raw[a]
        want = ref[a] - raw[a]
        assert np.abs(got - want).max() <= 1e-4 * np.abs(want).max(), a
    mv, lw = TO.activate(ref[0], ref[1])
    assert np.allclose(rend[0].cpu().numpy(), mv, rtol=1e-5, atol=1e-6)
    assert np.allclose(rend[1].cpu().numpy(), lw, rtol=1e-5, atol=1e-6)


def test_counted_adam_equals_host_step():
    """veg_adam_step_counted (step number on the device) takes the same
    steps as veg_adam_step, bit for bit, and advances its counter."""
    rng = np.random.default_rng(73)
    n = 2049
    raw = [rng.normal(0, 1, (n, 4)).astype(np.float32) for _ in range(5)]
    lr = rng.uniform(1e-3, 5e-2, (5, 4))
    runs = []
    for counted in (False, True):
        p = [dev(r) for r in raw]
        gr = [torch.zeros_like(t) for t in p]
        m = [torch.zeros_like(t) for t in p]
        v = [torch.zeros_like(t) for t in p]
        rend = [torch.zeros_like(p[0]), torch.zeros_like(p[1])]
        arrays = _lib.adam_arrays(p, gr, m, v, rend)
        counter = torch.zeros(2, dtype=torch.int64, device="cuda")
        grng = np.random.default_rng(74)
        for step in range(1, 6):
            for a in range(5):
                gr[a].copy_(dev(grng.normal(0, 1, (n, 4)).astype(np.float32)))
            if counted:
                _lib.veg_adam_step_counted(arrays, n, lr, counter)
            else:
                _lib.veg_adam_step(arrays, n, lr, step)
        torch.cuda.synchronize()
        runs.append([t.cpu().numpy() for t in p + m + v + rend])
        if counted:
            assert int(counter[0]) == 5
    for a, b in zip(*runs):
        assert np.array_equal(a, b)


def small_training_set(n=300, size=(48, 40), n_views=2, K=3, seed=74):
    bf = S.blob_field(4, seed)
    g, lt = S.initial_model(n, bf, seed + 1, weight=0.5)
    rng = np.random.default_rng(seed + 4)
    # visible at this small image size; anisotropic and rotated, so that every
    # gradient (the quaternion's included) is nontrivial
    g.logscale_w[:, :3] += 0.6 + rng.normal(0, 0.3, (n, 3)).astype(np.float32)
    q = rng.standard_normal((n, 4))
    g.quat[:] = (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)
    cams = S.grid_orbit_cameras(n_views, 1, size[0], size[1])
    luts = opacity_guided_luts(K, S.colour_ramp(seed + 2))
    tg = np.random.default_rng(seed + 3).uniform(0, 0.4, (n_views, K, size[1], size[0], 4))
    tg = tg.astype(np.float32)
    return g, lt, cams, luts, tg


def test_training_iteration_gradients_match_oracle():
    """One opacity-guided iteration (view 1, map 2): the loss and every
    accumulated gradient against the oracle's chain render -> L1 + SSIM ->
    composite backward -> projection and shading backward."""
    g, lt, cams, luts, tg = small_training_set()
    P = TrainParams(g, lt)
    T = OpacityGuidedTrainer(P, cams, lut_tensor(luts), dev(tg))
    T.step(view=1, k=2)
    torch.cuda.synchronize()
    cam, lut = cams[1], luts[2:3].astype(np.float64)
    d = lt.as_dict([O.headlight(cam)])
    proj, bins, fwd = O.render([cam], g, lut, record=True, lighting=d)
    assert not fwd["flag"].any()  # no threshold-straddling pixel in this scene
    loss, l1, ss, dout = TO.l1_ssim_loss(fwd["out"], tg[1, 2][None, None], 0.2)
    assert float(T.loss[0]) == pytest.approx(loss, rel=1e-4)
    g2 = O.composite_bwd(proj, [cam], bins, lut, (0, 0, 0), fwd, dout)
    gm, gl, gq = O.params_grad([cam], g, proj, g2)
    dn, dka, dkd, dks, db, dm = O.lighting_grad([cam], g, d, proj, g2)
    got = [x.cpu().numpy() for x in P.grads]

    def close(a, b, name):
        assert np.abs(a - b).max() <= 1e-3 * np.abs(b).max(), name

    close(got[0][:, :3], gm[:, :3] + dm, "mean")
    close(got[0][:, 3], gm[:, 3], "v")
    close(got[1][:, :3], gl[:, :3], "logscale")
    close(got[1][:, 3], gl[:, 3], "w")
    close(got[2], gq, "quat")
    close(got[3][:, :3], dn, "normal")
    close(got[3][:, 3], db, "beta")
    close(got[4][:, 0], dka, "k_a")
    close(got[4][:, 1], dkd, "k_d")
    close(got[4][:, 2], dks, "k_s")


def test_training_reduces_the_loss():
    """A model initialised from the volume learns targets rendered from a
    denser model of the same field under the opacity maps."""
    bf = S.blob_field(5, 75)
    gt, _ = S.field_gaussians(6000, 5, 75)
    cams = S.grid_orbit_cameras(8, 2, 64, 64, el_max_deg=30.0)
    luts = lut_tensor(opacity_guided_luts(4, S.colour_ramp(76)))
    from paper_2504_13339_gb300.render import SplatPipeline
    p = SplatPipeline(gt.n, cams, n_tf=4)
    tens = (dev(gt.mean_v), dev(gt.logscale_w), dev(gt.quat))
    p.render(*tens, luts)
    targets = p.out.clone()  # [V][K][H][W][4]
    g0, _ = S.initial_model(3000, bf, 77, weight=0.3, lighting=False)
    P = TrainParams(g0)
    T = OpacityGuidedTrainer(P, cams, luts, targets, seed=78)
    held = [(v, k) for v in range(0, 16, 3) for k in range(4)]
    eval0 = T.evaluate(held)
    losses = []
    for _ in range(300):
        T.step()
        losses.append(T.loss[0].clone())
    torch.cuda.synchronize()
    losses = torch.stack(losses).cpu().numpy()
    assert not T.overflowed()
    assert np.all(np.isfinite(losses))
    assert losses[-50:].mean() < 0.8 * losses[:50].mean(), (losses[:50].mean(),
                                                             losses[-50:].mean())
    eval1 = T.evaluate(held)
    assert eval1 < 0.8 * eval0, (eval0, eval1)


def test_evaluate_scores_a_pair_as_the_step_does():
    """evaluate() renders and scores a (view, map) pair as an iteration does
    before its update, and changes no parameter."""
    g, lt, cams, luts, tg = small_training_set(seed=96)
    P = TrainParams(g, lt)
    T = OpacityGuidedTrainer(P, cams, lut_tensor(luts), dev(tg))
    before = [x.clone() for x in P.raw]
    e = T.evaluate([(1, 2)])
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(before, P.raw))
    T.step(view=1, k=2)
    torch.cuda.synchronize()
    assert float(T.loss[0]) == pytest.approx(e, rel=1e-6)
    pair = [T.evaluate([(v, k)]) for v, k in ((0, 0), (1, 1))]
    assert T.evaluate([(0, 0), (1, 1)]) == pytest.approx(np.mean(pair), rel=1e-6)
    assert T.evaluate([]) != T.evaluate([])  # nan for no pairs


def test_native_step_equals_the_python_sequence():
    """veg_train_step issues the same stages as the Python sequence: the
    loss and every gradient of an iteration agree up to the order of the
    backward's float atomics, and the parameters after three iterations
    agree within two Adam steps (an element whose gradient is near zero may
    step either way when the summation order differs)."""
    from paper_2504_13339_gb300.train import default_lr
    g, lt, cams, luts, tg = small_training_set(seed=95)
    runs = []
    for native in (True, False):
        P = TrainParams(g, lt)
        T = OpacityGuidedTrainer(P, cams, lut_tensor(luts), dev(tg), native=native)
        T.step(view=0, k=1)
        torch.cuda.synchronize()
        first = (float(T.loss[0]), [x.cpu().numpy() for x in P.grads])
        for v, k in ((1, 2), (1, 0)):
            T.step(view=v, k=k)
        torch.cuda.synchronize()
        runs.append((first, [x.cpu().numpy() for x in P.raw]))
    ((la, ga), pa), ((lb, gb), pb) = runs
    assert la == pytest.approx(lb, rel=1e-6)
    for x, y in zip(ga, gb):
        assert np.abs(x - y).max() <= 1e-4 * np.abs(y).max()
    lr = default_lr()
    for a, (x, y) in enumerate(zip(pa, pb)):
        assert np.all(np.abs(x - y) <= 2 * 3 * lr[a][None, :] + 1e-6), a


def test_graph_replayed_training_step_matches_eager():
    """The whole training step (zeroing, project, bin, composite, L1, both
    backward passes, Adam with the device step counter) captured once as a
    CUDA graph and replayed takes the same three steps as the eager calls:
    losses within float32 summation-order noise, parameters within two Adam
    steps (the backward's float atomics may order sums differently)."""
    from paper_2504_13339_gb300.graphs import CapturedStep
    from paper_2504_13339_gb300.render import SplatPipeline
    from paper_2504_13339_gb300.train import default_lr
    g, lt, cams, luts, tg = small_training_set(seed=97)
    cams = cams[:1]
    lut = lut_tensor(luts[:2])
    target = dev(tg[:1, :2])
    lr = default_lr(lighting=False)
    runs = []
    for graphed in (False, True):
        P = TrainParams(g)
        P.use_device_counter()
        p = SplatPipeline(P.n, cams, n_tf=2)
        start = ([t.clone() for t in P.raw[:3]], [t.clone() for t in P.m[:3]],
                 [t.clone() for t in P.v[:3]], P.mean_v.clone(), P.logscale_w.clone())

        def step():
            P.zero_grad()
            p.project(P.mean_v, P.logscale_w, P.raw[2], lut)
            p.bin_sort()
            p.composite(lut)
            p.l1(target)
            p.backward_2d(p.loss_grad)
            p.project_backward(*P.grads[:3])
            P.adam(lr)
        losses = []
        if graphed:
            cs = CapturedStep(step)  # its two warm-up steps run eagerly: restore
            for dst, src in zip(P.raw[:3] + P.m[:3] + P.v[:3] + [P.mean_v, P.logscale_w],
                                start[0] + start[1] + start[2] + [start[3], start[4]]):
                dst.copy_(src)
            P.counter.zero_()
            for _ in range(3):
                cs.replay()
                losses.append(p.loss.clone())
        else:
            for _ in range(3):
                step()
                losses.append(p.loss.clone())
        torch.cuda.synchronize()
        assert int(P.counter[0]) == 3
        runs.append(([float(x) for x in losses], [t.cpu().numpy() for t in P.raw[:3]]))
    (la, pa), (lb, pb) = runs
    assert np.allclose(la, lb, rtol=1e-5)
    for a, (x, y) in enumerate(zip(pa, pb)):
        assert np.all(np.abs(x - y) <= 2 * 3 * lr[a][None, :] + 1e-6), a


def test_bucketed_projection_backward_is_bit_identical():
    """The projection backward split into Gaussian ranges (as the
    data-parallel step runs it, each range's all-reduce overlapping the
    next range) gives the same bits as one call, for several bucket counts,
    including one range per Gaussian at the tail; rows outside a range are
    left untouched; an out-of-range request is refused."""
    from paper_2504_13339_gb300 import parallel
    from paper_2504_13339_gb300.render import SplatPipeline
    g, lt, cams, luts, tg = small_training_set(seed=99)
    lut = lut_tensor(luts[:2])
    P = TrainParams(g)
    p = SplatPipeline(P.n, cams[:2], n_tf=2)
    p.project(P.mean_v, P.logscale_w, P.raw[2], lut)
    p.bin_sort()
    p.composite(lut)
    p.l1(dev(tg[:2, :2]))
    p.backward_2d(p.loss_grad)
    whole = [torch.zeros_like(t) for t in P.raw[:3]]
    p.project_backward(*whole)
    for nb in (1, 3, 7, P.n):
        parts = [torch.zeros_like(t) for t in P.raw[:3]]
        parallel.project_allreduce(p, parts, n_buckets=nb)
        for a, b in zip(whole, parts):
            assert torch.equal(a, b), nb
    # one range only: rows outside it stay as they were
    first, count = P.n // 3, P.n // 4
    sentinel = [torch.full_like(t, 7.0) for t in P.raw[:3]]
    for t in sentinel:
        t[first:first + count] = 0.0
    p.project_backward(*sentinel, first=first, count=count)
    for s, w in zip(sentinel, whole):
        assert bool((s[:first] == 7.0).all()) and bool((s[first + count:] == 7.0).all())
        assert torch.equal(s[first:first + count], w[first:first + count])
    with pytest.raises(_lib.VegError):
        p.project_backward(*sentinel, first=P.n - 2, count=3)
    with pytest.raises(_lib.VegError):
        p.project_backward(*sentinel, first=-1, count=2)
