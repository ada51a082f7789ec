"""Volume raymarching oracle: the ground-truth renderer of the paper's
training data, stated plainly in float64 on the CPU.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA library and never calls it.

What it computes.  The paper trains from images that a volume renderer
"raymarches ... with an emission-absorption model and shades ... with
Blinn-Phong lighting with a headlight from the camera" (Sec. 4.2, 5.1).  This
oracle marches each pixel's ray through a scalar volume on a regular grid,
maps every sample through the transfer function, shades it and composites
front to back.

Readings (the paper names the renderer, not its parameters; listed in the
design notes):
  R24 volume: R^3 vertex values at x_i = -1 + 2 i/(R-1) on each axis, layout
      [z][y][x]; the value at a point of [-1,1]^3 is the trilinear
      interpolation of its cell's eight vertices.  The gradient is, as volume
      renderers precompute it, central differences at the vertices
      ((v[i+1] - v[i-1]) / 2h; one-sided (v[1] - v[0]) / h and
      (v[R-1] - v[R-2]) / h on the boundary faces) interpolated trilinearly
      like the value, so it is continuous across cells.
  R25 rays: the camera model of the splatting path (pinhole, OpenCV axes,
      pixel (i, j) at the point (i, j)); direction d = normalised R^T
      ((i - cx)/fx, (j - cy)/fy, 1) from the camera centre; the ray is
      clipped to the box [-1,1]^3 (slab test) and to t >= near; with
      [t0, t1] the clipped interval and step Delta, samples sit at
      t0 + (k + 1/2) Delta for k = 0 .. floor((t1 - t0)/Delta) - 1.
  R26 emission-absorption: a sample's opacity is alpha = 1 - (1 - A(v))^(Delta/h)
      with h the grid spacing (A is the opacity per unit distance h, the
      convention of VTK's scalar opacity unit distance); colour C(v); both
      from the transfer function tables (reading R6's interpolation).
  R27 shading: Blinn-Phong with global k_a, k_d, k_s, beta, the normal
      n = -grad/|grad|, l = headlight (the camera's backward optical axis),
      e = -d, h = (e + l)/|e + l|: c = (k_a + k_d |n.l|) C(v) + k_s |n.h|^beta
      (specular 0 where n.l = 0).  Where the gradient vanishes there is no
      normal and only the ambient term remains: c = k_a C(v).
  R28 compositing: front to back, C += T alpha c, T *= 1 - alpha; the ray
      stops after the sample that brings T below 1e-4.  Output (C + T bg, T).
  Flags (for float32 comparisons): a pixel is flagged when its sample count
  floor((t1 - t0)/Delta) has a fraction within 1e-3 of an integer or when a
  transmittance comes within a relative 1e-3 of 1e-4.
"""
from __future__ import annotations

import numpy as np

T_STOP = 1e-4


def camera_ray(cam, i, j):
    w2c = np.asarray(cam.world_to_cam, np.float64)
    R, t = w2c[:, :3], w2c[:, 3]
    eye = -R.T @ t
    dc = np.array([(i - cam.cx) / cam.fx, (j - cam.cy) / cam.fy, 1.0])
    d = R.T @ dc
    return eye, d / np.linalg.norm(d)


def clip_box(eye, d, near):
    """[t0, t1] of the ray inside [-1,1]^3 and t >= near (None if empty)."""
    t0, t1 = near, np.inf
    for a in range(3):
        if d[a] == 0.0:
            if abs(eye[a]) > 1.0:
                return None
            continue
        ta, tb = (-1.0 - eye[a]) / d[a], (1.0 - eye[a]) / d[a]
        t0 = max(t0, min(ta, tb))
        t1 = min(t1, max(ta, tb))
    return (t0, t1) if t1 > t0 else None


def vertex_gradients(vol):
    """(R, R, R, 3) gradient (d/dx, d/dy, d/dz) at every vertex: central
    differences inside, one-sided on the boundary faces (reading R24)."""
    v = np.asarray(vol, np.float64)
    R = v.shape[0]
    h = 2.0 / (R - 1)
    out = np.zeros(v.shape + (3,))
    for comp, axis in ((0, 2), (1, 1), (2, 0)):  # x is the last array axis
        d = np.zeros_like(v)
        sl = lambda a, b: tuple(slice(a, b) if ax == axis else slice(None) for ax in range(3))
        d[sl(1, R - 1)] = (v[sl(2, R)] - v[sl(0, R - 2)]) / (2 * h)
        d[sl(0, 1)] = (v[sl(1, 2)] - v[sl(0, 1)]) / h
        d[sl(R - 1, R)] = (v[sl(R - 1, R)] - v[sl(R - 2, R - 1)]) / h
        out[..., comp] = d
    return out


def trilinear(vol, p, grads=None):
    """Value and gradient (d/dx, d/dy, d/dz) at p in [-1,1]^3: trilinear
    interpolation of the vertex values and of the vertex gradients
    (vertex_gradients(vol) unless given); vol[z][y][x]."""
    R = vol.shape[0]
    h = 2.0 / (R - 1)
    if grads is None:
        grads = vertex_gradients(vol)
    g = (np.asarray(p, np.float64) + 1.0) / h  # grid coordinates (x, y, z)
    i = np.clip(np.floor(g).astype(int), 0, R - 2)
    f = g - i
    x0, y0, z0 = i
    c = vol[z0:z0 + 2, y0:y0 + 2, x0:x0 + 2].astype(np.float64)  # [z][y][x]
    cg = grads[z0:z0 + 2, y0:y0 + 2, x0:x0 + 2]
    fx, fy, fz = f
    wx = np.array([1 - fx, fx])
    wy = np.array([1 - fy, fy])
    wz = np.array([1 - fz, fz])
    val = np.einsum("zyx,z,y,x->", c, wz, wy, wx)
    grad = np.einsum("zyxc,z,y,x->c", cg, wz, wy, wx)
    return val, grad


def tf_lookup(lut, v):
    """Reading R6: linear interpolation of an L-entry table over [0, 1]."""
    L = lut.shape[0]
    p = min(max(v, 0.0), 1.0) * (L - 1)
    k = min(int(np.floor(p)), L - 2)
    tau = p - k
    return (1.0 - tau) * lut[k] + tau * lut[k + 1]


def march_pixel(cam, vol, luts, i, j, step, material=None, bg=(0.0, 0.0, 0.0)):
    """(T, 4) output of pixel (i, j) for every table; also the per-table
    transmittance just before each sample's stop test for flagging."""
    luts = np.asarray(luts, np.float64)
    nT = luts.shape[0]
    R = vol.shape[0]
    h = 2.0 / (R - 1)
    eye, d = camera_ray(cam, i, j)
    C = np.zeros((nT, 3))
    T = np.ones(nT)
    live = np.ones(nT, bool)
    near_stop = np.zeros(nT, bool)
    seg = clip_box(eye, d, cam.near)
    grads = vertex_gradients(vol) if material is not None else np.zeros(vol.shape + (3,))
    if seg is not None:
        t0, t1 = seg
        n = int(np.floor((t1 - t0) / step))
        frac = (t1 - t0) / step - n
        if frac < 1e-3 or frac > 1.0 - 1e-3:
            near_stop[:] = True
        w2c = np.asarray(cam.world_to_cam, np.float64)
        light = -w2c[2, :3]
        e = -d
        hv = (e + light) / np.linalg.norm(e + light)
        for k in range(n):
            if not live.any():
                break
            p = eye + (t0 + (k + 0.5) * step) * d
            v, g = trilinear(vol, p, grads)
            shade = None
            if material is not None:
                gn = np.linalg.norm(g)
                ka, kd, ks, beta = material
                if gn > 0.0:
                    nrm = -g / gn
                    nl = abs(nrm @ light)
                    sd = ka + kd * nl
                    ss = ks * abs(nrm @ hv) ** beta if nl > 0 else 0.0
                    shade = (sd, ss)
                else:
                    shade = (ka, 0.0)
            for t in range(nT):
                if not live[t]:
                    continue
                rgba = tf_lookup(luts[t], v)
                alpha = 1.0 - (1.0 - rgba[3]) ** (step / h)
                col = rgba[:3] if shade is None else shade[0] * rgba[:3] + shade[1]
                C[t] += T[t] * alpha * col
                T[t] *= 1.0 - alpha
                if abs(T[t] / T_STOP - 1.0) < 1e-3:
                    near_stop[t] = True
                if T[t] < T_STOP:
                    live[t] = False
    out = np.concatenate([C + T[:, None] * np.asarray(bg, np.float64)[None], T[:, None]], 1)
    return out, near_stop


def render(cam, vol, luts, step, material=None, bg=(0.0, 0.0, 0.0), pixels=None):
    """Image [T][H][W][4] (or only the listed (i, j) pixels) and the flags of
    pixels whose stop decision sits within 1e-3 of T = 1e-4."""
    luts = np.asarray(luts, np.float64)
    nT = luts.shape[0]
    out = np.zeros((nT, cam.height, cam.width, 4))
    out[..., :3] = np.asarray(bg)
    out[..., 3] = 1.0
    flag = np.zeros((nT, cam.height, cam.width), bool)
    pix = [(i, j) for j in range(cam.height) for i in range(cam.width)] if pixels is None \
        else pixels
    for i, j in pix:
        o, f = march_pixel(cam, vol, luts, i, j, step, material, bg)
        out[:, j, i] = o
        flag[:, j, i] = f
    return out, flag
