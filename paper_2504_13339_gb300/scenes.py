"""Seeded synthetic inputs for the VEG splatting path.

This module draws random numbers and describes cameras, transfer functions and
Gaussian scenes.  It holds none of the rendering method's arithmetic: both the
CUDA path and the CPU oracle consume exactly these arrays.

Conventions (the paper leaves them open, Sec. 3.3):
  * cameras are pinholes with OpenCV axes (x right, y down, z forward); the
    world-to-camera transform is a rigid 3x4 row-major [R | t];
  * focal length f = W / (2 tan(fov/2)) on both axes, principal point
    ((W-1)/2, (H-1)/2), so pixel (i, j) is evaluated at the point (i, j);
  * a Gaussian is three float4 rows: (mu_x, mu_y, mu_z, v), (log s_x, log s_y,
    log s_z, w), (q_w, q_x, q_y, q_z); v and w are already activated to [0, 1]
    (the paper stores them through a sigmoid, Sec. 3.3);
  * a transfer function is a 256-entry RGBA table over v in [0, 1] with
    straight (not premultiplied) colour and opacity in the alpha channel.

Scene recipes follow the workloads of the paper's evaluation (Sec. 5.1):
scalar-valued Gaussians whose means sample a volume, with transfer functions
made of opacity bumps; the paper's datasets are replaced by sums of random
anisotropic 3D Gaussian blobs ("blob fields").
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LUT_SIZE = 256
NEAR = 0.2


@dataclass
class Camera:
    world_to_cam: np.ndarray  # (3, 4) float32, row-major [R | t]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = NEAR
    meta: dict = field(default_factory=dict)

    @property
    def tiles_x(self) -> int:
        return (self.width + 15) // 16

    @property
    def tiles_y(self) -> int:
        return (self.height + 15) // 16


def look_at_camera(eye, width, height, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0),
                   fov_deg=45.0, near=NEAR) -> Camera:
    """Pinhole camera at `eye` looking at `target`, world `up` shown upwards."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    rot = np.stack([right, down, fwd])
    t = -rot @ eye
    w2c = np.concatenate([rot, t[:, None]], axis=1).astype(np.float32)
    f = width / (2.0 * math.tan(math.radians(fov_deg) / 2.0))
    return Camera(w2c, float(np.float32(f)), float(np.float32(f)),
                  (width - 1) / 2.0, (height - 1) / 2.0, int(width), int(height), near,
                  {"eye": eye.tolist(), "fov_deg": fov_deg})


def orbit_camera(azimuth_deg, elevation_deg, radius, width, height, fov_deg=45.0) -> Camera:
    az, el = math.radians(azimuth_deg), math.radians(elevation_deg)
    eye = radius * np.array([math.sin(az) * math.cos(el), math.sin(el),
                             math.cos(az) * math.cos(el)])
    return look_at_camera(eye, width, height, fov_deg=fov_deg)


def orbit_cameras(n, seed, width, height, radius=3.0, el_max_deg=30.0) -> list[Camera]:
    """`n` views on a radius-`radius` orbit: azimuth uniform, elevation in +-el_max."""
    rng = np.random.default_rng(seed)
    az = rng.uniform(0.0, 360.0, n)
    el = rng.uniform(-el_max_deg, el_max_deg, n)
    return [orbit_camera(a, e, radius, width, height) for a, e in zip(az, el)]


def grid_orbit_cameras(n_az, n_el, width, height, radius=3.0, el_max_deg=60.0) -> list[Camera]:
    """A training orbit like the paper's (Sec. 5.1: 16 azimuths x 10
    elevations): azimuths k 360/n_az, elevations evenly spaced in
    [-el_max, el_max]."""
    els = np.linspace(-el_max_deg, el_max_deg, n_el) if n_el > 1 else np.zeros(1)
    return [orbit_camera(360.0 * a / n_az, float(e), radius, width, height)
            for e in els for a in range(n_az)]


def camera_array(cams) -> np.ndarray:
    """Pack cameras as float32 rows of 16: w2c(12), fx, fy, cx, cy."""
    rows = []
    for c in cams:
        rows.append(np.concatenate([c.world_to_cam.reshape(12),
                                    np.array([c.fx, c.fy, c.cx, c.cy], np.float32)]))
    return np.stack(rows).astype(np.float32)


# ----------------------------------------------------------------------------
# Gaussians
# ----------------------------------------------------------------------------

@dataclass
class Gaussians:
    mean_v: np.ndarray       # (N, 4) float32: mu, v
    logscale_w: np.ndarray   # (N, 4) float32: log-scale, w
    quat: np.ndarray         # (N, 4) float32: q_w, q_x, q_y, q_z

    @property
    def n(self) -> int:
        return self.mean_v.shape[0]

    def copy(self) -> "Gaussians":
        return Gaussians(self.mean_v.copy(), self.logscale_w.copy(), self.quat.copy())

    def subset(self, idx) -> "Gaussians":
        return Gaussians(self.mean_v[idx].copy(), self.logscale_w[idx].copy(),
                         self.quat[idx].copy())


def _random_quats(rng, n) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def uniform_gaussians(n, seed, logscale_mean=-3.5, logscale_std=0.3, weight=1.0) -> Gaussians:
    """Means uniform in [-1,1]^3, log-scales N(mean, std) per axis, random unit
    quaternions, scalars U[0,1], weights `weight` (the small plain-render scene)."""
    rng = np.random.default_rng(seed)
    mean = rng.uniform(-1.0, 1.0, (n, 3))
    v = rng.uniform(0.0, 1.0, (n, 1))
    ls = rng.normal(logscale_mean, logscale_std, (n, 3))
    w = np.full((n, 1), weight)
    q = _random_quats(rng, n)
    return Gaussians(np.concatenate([mean, v], 1).astype(np.float32),
                     np.concatenate([ls, w], 1).astype(np.float32), q)


@dataclass
class BlobField:
    amp: np.ndarray      # (K,)
    center: np.ndarray   # (K, 3)
    rot: np.ndarray      # (K, 3, 3)
    sigma: np.ndarray    # (K, 3)

    def value(self, pts: np.ndarray, chunk=1 << 20) -> np.ndarray:
        """Field value sum_k a_k exp(-1/2 (x-m_k)^T S_k^-1 (x-m_k)) in float64."""
        pts = np.asarray(pts, np.float64)
        out = np.zeros(pts.shape[0])
        for s in range(0, pts.shape[0], chunk):
            p = pts[s:s + chunk]
            acc = np.zeros(p.shape[0])
            for k in range(self.amp.shape[0]):
                d = (p - self.center[k]) @ self.rot[k]  # coordinates in blob frame
                q = ((d / self.sigma[k]) ** 2).sum(1)
                acc += self.amp[k] * np.exp(-0.5 * q)
            out[s:s + chunk] = acc
        return out


def field_gradient(bf, pts, chunk=1 << 20) -> np.ndarray:
    """Gradient of the blob field at `pts` (N, 3), float64:
    sum_k -a_k exp(-q_k/2) S_k^-1 (x - m_k) with S_k^-1 = R_k diag(1/sigma^2) R_k^T."""
    pts = np.asarray(pts, np.float64)
    out = np.zeros_like(pts)
    for s in range(0, pts.shape[0], chunk):
        p = pts[s:s + chunk]
        acc = np.zeros_like(p)
        for k in range(bf.amp.shape[0]):
            d = (p - bf.center[k]) @ bf.rot[k]
            e = bf.amp[k] * np.exp(-0.5 * ((d / bf.sigma[k]) ** 2).sum(1))
            acc -= e[:, None] * ((d / bf.sigma[k] ** 2) @ bf.rot[k].T)
        out[s:s + chunk] = acc
    return out


def gradient_lighting(g: "Gaussians", bf, ka=0.3, kd=0.7, ks=0.2, beta=20.0) -> "Lighting":
    """Lighting whose normals follow the field (the negated, normalised
    gradient at each mean, as a volume renderer shades by the gradient)."""
    gr = field_gradient(bf, g.mean_v[:, :3])
    nrm = -gr / np.maximum(np.linalg.norm(gr, axis=1, keepdims=True), 1e-12)
    nb = np.concatenate([nrm, np.full((g.n, 1), beta)], 1).astype(np.float32)
    k = np.tile(np.array([ka, kd, ks, 0.0], np.float32), (g.n, 1))
    return Lighting(nb, k)


def field_volume(bf, R) -> np.ndarray:
    """The blob field sampled at the R^3 vertices x_i = -1 + 2i/(R-1),
    layout [z][y][x], normalised by its largest vertex value (float32): the
    gridded volume of a structured dataset."""
    x = np.linspace(-1.0, 1.0, R)
    out = np.empty((R, R, R), np.float32)
    Y, X = np.meshgrid(x, x, indexing="ij")
    for k in range(R):  # one z slice at a time
        pts = np.stack([X.ravel(), Y.ravel(), np.full(X.size, x[k])], 1)
        out[k] = bf.value(pts).reshape(R, R)
    return (out / out.max()).astype(np.float32)


def blob_field(n_blobs, seed) -> BlobField:
    rng = np.random.default_rng(seed)
    amp = rng.uniform(0.3, 1.0, n_blobs)
    center = rng.uniform(-0.7, 0.7, (n_blobs, 3))
    sigma = rng.uniform(0.08, 0.35, (n_blobs, 3))
    rot = []
    for _ in range(n_blobs):
        a = rng.standard_normal((3, 3))
        qm, r = np.linalg.qr(a)
        qm *= np.sign(np.diag(r))
        if np.linalg.det(qm) < 0:
            qm[:, 0] = -qm[:, 0]
        rot.append(qm)
    return BlobField(amp, center, np.stack(rot), sigma)


def field_gaussians(n, n_blobs, seed, logscale_std=0.3, weight=1.0):
    """`n` Gaussians whose means are drawn from the density proportional to a
    blob field on [-1,1]^3 (exact mixture sampling with rejection outside the
    cube), scalar = field value at the mean normalised by its sample maximum,
    log-scale N(ln(0.5 * 2 / n^(1/3)), std) per axis (half the mean spacing of
    n points in the cube).  Returns (Gaussians, BlobField)."""
    bf = blob_field(n_blobs, seed)
    rng = np.random.default_rng(seed + 7919)
    mass = bf.amp * np.prod(bf.sigma, axis=1)
    prob = mass / mass.sum()
    pts = np.empty((0, 3))
    while pts.shape[0] < n:
        m = int((n - pts.shape[0]) * 1.3) + 1024
        k = rng.choice(n_blobs, size=m, p=prob)
        z = rng.standard_normal((m, 3)) * bf.sigma[k]
        x = np.einsum("mij,mj->mi", bf.rot[k], z) + bf.center[k]
        x = x[np.all(np.abs(x) <= 1.0, axis=1)]
        pts = np.concatenate([pts, x])
    pts = pts[:n]
    f = bf.value(pts)
    v = np.clip(f / f.max(), 0.0, 1.0)
    mu_ls = math.log(0.5 * 2.0 / n ** (1.0 / 3.0))
    ls = rng.normal(mu_ls, logscale_std, (n, 3))
    q = _random_quats(rng, n)
    g = Gaussians(np.concatenate([pts, v[:, None]], 1).astype(np.float32),
                  np.concatenate([ls, np.full((n, 1), weight)], 1).astype(np.float32), q)
    return g, bf


def perturbed(g: Gaussians, seed, mean_sigma=0.01, v_sigma=0.05) -> Gaussians:
    """Copy with means + N(0, mean_sigma^2) and scalars + N(0, v_sigma^2) clamped to [0,1]."""
    rng = np.random.default_rng(seed)
    out = g.copy()
    out.mean_v[:, :3] += rng.normal(0.0, mean_sigma, (g.n, 3)).astype(np.float32)
    out.mean_v[:, 3] = np.clip(out.mean_v[:, 3] + rng.normal(0.0, v_sigma, g.n), 0.0, 1.0)
    return out


# ----------------------------------------------------------------------------
# Transfer functions
# ----------------------------------------------------------------------------

def bump_tf(seed, n_bumps=3, peak=0.8, size=LUT_SIZE) -> np.ndarray:
    """RGBA table: opacity = peak * max_k exp(-(x-b_k)^2 / (2 w_k^2)) with
    b_k ~ U[0.1, 0.9], w_k ~ U[0.03, 0.1]; colour piecewise linear through four
    random colours at x = 0, 1/3, 2/3, 1."""
    rng = np.random.default_rng(seed)
    b = rng.uniform(0.1, 0.9, n_bumps)
    w = rng.uniform(0.03, 0.1, n_bumps)
    cols = rng.uniform(0.0, 1.0, (4, 3))
    x = np.arange(size) / (size - 1)
    op = peak * np.max(np.exp(-((x[:, None] - b[None]) ** 2) / (2 * w[None] ** 2)), axis=1)
    knots = np.linspace(0.0, 1.0, 4)
    rgb = np.stack([np.interp(x, knots, cols[:, c]) for c in range(3)], 1)
    return np.concatenate([rgb, op[:, None]], 1).astype(np.float32)


def colour_ramp(seed, size=LUT_SIZE) -> np.ndarray:
    """(size, 3) colours piecewise linear through four random colours at
    x = 0, 1/3, 2/3, 1 (a sequential stand-in for the colormap of the
    paper's training renders; no named colormap table is used)."""
    rng = np.random.default_rng(seed)
    cols = np.sort(rng.uniform(0.0, 1.0, (4, 3)), axis=0)  # monotone: not diverging
    x = np.arange(size) / (size - 1)
    knots = np.linspace(0.0, 1.0, 4)
    return np.stack([np.interp(x, knots, cols[:, c]) for c in range(3)], 1).astype(np.float32)


def bump_tfs(n, seed, **kw) -> np.ndarray:
    return np.stack([bump_tf(seed * 1000 + i, **kw) for i in range(n)])


def constant_tf(rgba, size=LUT_SIZE) -> np.ndarray:
    return np.tile(np.asarray(rgba, np.float32)[None], (size, 1))


@dataclass
class Lighting:
    """Per-Gaussian Blinn-Phong parameters (Eq. 2-3) in the library's packed
    layouts: normal_beta (N, 4) = (normal, beta), k_ads (N, 4) = (k_a, k_d,
    k_s, 0)."""
    normal_beta: np.ndarray
    k_ads: np.ndarray

    def as_dict(self, lights) -> dict:
        """The oracle's form: normal, ka, kd, ks, beta in float64 plus the
        per-view light directions."""
        nb = self.normal_beta.astype(np.float64)
        k = self.k_ads.astype(np.float64)
        return {"normal": nb[:, :3], "beta": nb[:, 3], "ka": k[:, 0], "kd": k[:, 1],
                "ks": k[:, 2], "lights": np.asarray(lights, np.float64)}


def random_lighting(n, seed, beta=(1.0, 30.0)) -> Lighting:
    """Normals N(0, I) (not normalised), k_a U[0.1, 0.6], k_d U[0.2, 0.9],
    k_s U[0, 0.8], shininess U[beta]."""
    rng = np.random.default_rng(seed)
    normal = rng.standard_normal((n, 3))
    ka = rng.uniform(0.1, 0.6, n)
    kd = rng.uniform(0.2, 0.9, n)
    ks = rng.uniform(0.0, 0.8, n)
    b = rng.uniform(beta[0], beta[1], n)
    nb = np.concatenate([normal, b[:, None]], 1).astype(np.float32)
    k = np.stack([ka, kd, ks, np.zeros(n)], 1).astype(np.float32)
    return Lighting(nb, k)


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------

def plain_scene(seed=1):
    """4096 Gaussians, one bump TF, camera at radius 3, 128x128, black background."""
    g = uniform_gaussians(4096, seed)
    cam = look_at_camera((0.0, 0.0, 3.0), 128, 128)
    tf = bump_tf(seed + 100)[None]
    return g, [cam], tf


def initial_model(n, bf: "BlobField", seed, weight=0.1, lighting=True):
    """A model to train (Sec. 4.1): `n` points drawn at random from the
    volume (uniform in the cube, as data points of a regular grid would be),
    each a Gaussian with the field's value there, log-scales from the mean
    spacing (reading R14), identity rotations, weight `weight`; with
    `lighting`, random unit normals, k_a 0.3, k_d 0.6, k_s 0.2, shininess 10.
    Returns (Gaussians, Lighting or None)."""
    rng = np.random.default_rng(seed)
    pts = rng.uniform(-1.0, 1.0, (n, 3))
    f = bf.value(pts)
    v = np.clip(f / f.max(), 0.0, 1.0)
    mu_ls = math.log(0.5 * 2.0 / n ** (1.0 / 3.0))
    ls = np.full((n, 3), mu_ls)
    q = np.tile(np.array([1.0, 0.0, 0.0, 0.0]), (n, 1))
    g = Gaussians(np.concatenate([pts, v[:, None]], 1).astype(np.float32),
                  np.concatenate([ls, np.full((n, 1), weight)], 1).astype(np.float32),
                  q.astype(np.float32))
    lt = None
    if lighting:
        nrm = rng.standard_normal((n, 3))
        nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
        nb = np.concatenate([nrm, np.full((n, 1), 10.0)], 1).astype(np.float32)
        k = np.tile(np.array([0.3, 0.6, 0.2, 0.0], np.float32), (n, 1))
        lt = Lighting(nb, k)
    return g, lt


def vertex_model(vol, n, seed, weight=0.1, lighting=True):
    """The paper's initialisation (Sec. 4.1): `n` vertices of the gridded
    volume drawn at random without replacement (connectivity dropped), each a
    Gaussian at the vertex carrying its value; scales from the mean spacing
    of n points (reading R14), identity rotations, weight `weight`; lighting
    as in initial_model.  Returns (Gaussians, Lighting or None)."""
    R = vol.shape[0]
    rng = np.random.default_rng(seed)
    idx = rng.choice(R ** 3, size=n, replace=False)
    z, y, x = np.unravel_index(idx, (R, R, R))
    grid = np.linspace(-1.0, 1.0, R)
    pts = np.stack([grid[x], grid[y], grid[z]], 1)
    v = vol.reshape(-1)[idx].astype(np.float64)
    mu_ls = math.log(0.5 * 2.0 / n ** (1.0 / 3.0))
    g = Gaussians(np.concatenate([pts, v[:, None]], 1).astype(np.float32),
                  np.concatenate([np.full((n, 3), mu_ls), np.full((n, 1), weight)], 1)
                  .astype(np.float32),
                  np.tile(np.array([1.0, 0.0, 0.0, 0.0], np.float32), (n, 1)))
    lt = None
    if lighting:
        nrm = rng.standard_normal((n, 3))
        nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
        nb = np.concatenate([nrm, np.full((n, 1), 10.0)], 1).astype(np.float32)
        lt = Lighting(nb, np.tile(np.array([0.3, 0.6, 0.2, 0.0], np.float32), (n, 1)))
    return g, lt


def train_scene(n=1_000_000, n_blobs=8, width=1024, n_tf=4, seed=2):
    """Training-step workload: blob-field Gaussians, a target made from a
    perturbed copy, `n_tf` bump TFs, one orbit view."""
    g, bf = field_gaussians(n, n_blobs, seed)
    target_g = perturbed(g, seed + 1)
    cam = orbit_camera(30.0, 20.0, 3.0, width, width)
    tfs = bump_tfs(n_tf, seed + 2)
    return g, target_g, [cam], tfs
