"""VEG splatting oracle: a plain, slow CPU statement of the rendering path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA library and never calls it.

What it computes (paper: Volume Encoding Gaussians, Sec. 3.3):
  * Eq. 1 -- front-to-back alpha blending  P = sum_i c_i a_i prod_{j<i} (1 - a_j);
  * the 3D covariance from scale and rotation and its EWA projection to a
    2D screen covariance (Sec. 3.3, "method of Zwicker et al.");
  * transfer-function mapping applied first, with linear interpolation between
    control points (Sec. 3.3, last paragraph), opacity a_i = O(v_i) * w_i;
  * the tile rasteriser of 3D Gaussian splatting the paper adopts: 16x16 tiles,
    per-tile lists in (tile, depth) order, per-pixel evaluation of the 2D
    Gaussian;
  * the manual backward pass through the rasteriser, the transfer function
    and the projection (Sec. 3.3).

Readings where the paper is silent (each listed in the design notes):
  R1 camera: OpenCV axes, f = W/(2 tan(fov/2)), principal point ((W-1)/2, (H-1)/2).
  R2 projection: +0.3 px^2 on the 2D covariance diagonal, x/z and y/z clamped
     to 1.3 tan(fov/2) inside the Jacobian, near cull at z <= 0.2, cull on a
     non-positive determinant, radius ceil(3 sqrt(lambda_max)) with
     lambda_max = m + sqrt(max(0.1, m^2 - det)).
  R3 binning-critical values (depth, screen mean, radius, tile rectangle, the
     opacity cull) are evaluated in IEEE float32 in the fixed operation order
     written in ``project32`` (every product and sum rounded separately, no
     fused multiply-add); everything after binning is float64.
  R4 ties in depth are broken by Gaussian index.
  R5 a Gaussian is culled before binning when A_t(v) w < 1/255 for every
     transfer function t of the call (lossless: its alpha can never reach
     1/255 since the 2D Gaussian is <= 1).
  R6 transfer function: N entries at x_k = k/(N-1); p = clamp(v,0,1)(N-1),
     k = min(floor(p), N-2), tau = p - k, value = (1-tau) L[k] + tau L[k+1];
     d/dv = (N-1)(L[k+1]-L[k]) for v in [0,1], else 0.
  R7 skip a pair when power > 0 or alpha < 1/255; alpha = min(0.99, A w G);
     stop a pixel (per transfer function) when T (1-alpha) < 1e-4, without
     blending that splat.
  R8 output RGB = sum c a T + T_final bg and the final transmittance T_final.
  R9 derivatives are the true ones: zero through the 0.99 clamp and the skips.
  R12 pixels whose decisions sit within a relative 1e-5 (alpha tests) or 1e-3
     (transmittance stop) of a threshold, or whose exponent is zero to within
     1e-5 of its terms, are flagged; float32 and float64 may legitimately
     decide them differently.  ``pixel_alternatives`` lists every outcome of
     such a pixel (each flagged decision taken both ways), so a flagged pixel
     is checked against the outcome with the same decisions, not dropped.
"""
from __future__ import annotations

import math

import numpy as np

F = np.float32

ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_MIN = 1e-4
DILATION = 0.3
FRUSTUM_SLACK = 1.3
LAMBDA_FLOOR = 0.1
TILE = 16
# Relative half-widths of the threshold windows of reading R12.  Float32
# alpha carries up to a few 1e-6 relative error (the exponent's rounding
# times |power| <= ~6, plus the hardware exp2 approximation); float32
# transmittance accumulates up to ~1e-5 per high-opacity step.
FLAG_ALPHA = 1e-5
FLAG_T = 1e-3

# Cody-Waite split of ln 2: the high part has 15 significant bits so that
# n * LN2_HI is exact for |n| <= 2^8; LN2_LO = ln 2 - LN2_HI.
_LN2_HI = F(0.693145751953125)
_LN2_LO = F(1.4286068203094172e-06)
_LOG2E = F(1.4426950408889634)


# ============================================================================
# float32 section (binning-critical values, reading R3)
# ============================================================================

def exp32(x):
    """exp in float32 by Cody-Waite argument reduction and a degree-7 Taylor
    polynomial in Horner form (Cody & Waite, "Software Manual for the
    Elementary Functions", 1980).  Every operation is one rounded float32 op.
    Input clamped to [-80, 80]."""
    x = np.minimum(np.maximum(np.asarray(x, F), F(-80.0)), F(80.0))
    n = np.rint(x * _LOG2E).astype(F)
    r = (x - n * _LN2_HI).astype(F)
    r = (r - n * _LN2_LO).astype(F)
    p = F(1.0 / 5040.0)
    for c in (1.0 / 720.0, 1.0 / 120.0, 1.0 / 24.0, 1.0 / 6.0, 0.5, 1.0, 1.0):
        p = (p * r).astype(F)
        p = (p + F(c)).astype(F)
    ni = n.astype(np.int32)
    scale = ((ni + 127).astype(np.uint32) << np.uint32(23)).view(F)
    return (p * scale).astype(F)


def tf_eval32(lut, v):
    """Linear interpolation of a (L, C) float32 table at v (reading R6), float32."""
    lut = np.asarray(lut, F)
    L = lut.shape[0]
    v = np.asarray(v, F)
    vc = np.minimum(np.maximum(v, F(0.0)), F(1.0))
    p = (vc * F(L - 1)).astype(F)
    k = np.minimum(np.floor(p), F(L - 2)).astype(np.int64)
    tau = (p - k.astype(F)).astype(F)
    one_m = (F(1.0) - tau).astype(F)
    lo = lut[k]
    hi = lut[k + 1]
    a = (one_m[..., None] * lo).astype(F)
    b = (tau[..., None] * hi).astype(F)
    return (a + b).astype(F)


def _dot3(a0, a1, a2, b0, b1, b2):
    return ((a0 * b0 + a1 * b1).astype(F) + a2 * b2).astype(F)


def project32(cam, g, luts=None):
    """Per-Gaussian projection in float32 (Sec. 3.3 + readings R1-R5).

    The operation order below is the specification of the binning-critical
    arithmetic; every line is one rounded float32 operation.  Returns a dict
    with geo (N,4) = (u_x, u_y, depth, w), aux (N,4) = (conic a, b, c, v),
    count (N,) tiles touched, rect (N,4) = (x0, y0, x1, y1) in tiles (end
    exclusive), all zero for culled Gaussians.
    """
    with np.errstate(all="ignore"):
        return _project32(cam, g, luts)


def _project32(cam, g, luts):
    n = g.n
    w2c = np.asarray(cam.world_to_cam, F)
    r = [[w2c[i, j] for j in range(3)] for i in range(3)]
    tv = [w2c[i, 3] for i in range(3)]
    fx, fy, cx, cy = F(cam.fx), F(cam.fy), F(cam.cx), F(cam.cy)
    W, H = cam.width, cam.height
    mx, my, mz, v = (g.mean_v[:, i].astype(F) for i in range(4))
    lx, ly, lz, wt = (g.logscale_w[:, i].astype(F) for i in range(4))
    qw, qx, qy, qz = (g.quat[:, i].astype(F) for i in range(4))

    # camera-space position
    t = [(_dot3(r[i][0], r[i][1], r[i][2], mx, my, mz) + tv[i]).astype(F) for i in range(3)]
    tx, ty, tz = t
    ok = tz > F(cam.near)
    inv_z = (F(1.0) / tz).astype(F)
    xr = (tx * inv_z).astype(F)
    yr = (ty * inv_z).astype(F)
    ux = ((fx * xr).astype(F) + cx).astype(F)
    uy = ((fy * yr).astype(F) + cy).astype(F)
    limx = (F(FRUSTUM_SLACK) * ((F(0.5) * F(W)).astype(F) / fx).astype(F)).astype(F)
    limy = (F(FRUSTUM_SLACK) * ((F(0.5) * F(H)).astype(F) / fy).astype(F)).astype(F)
    xc = np.minimum(np.maximum(xr, -limx), limx)
    yc = np.minimum(np.maximum(yr, -limy), limy)
    j00 = (fx * inv_z).astype(F)
    j11 = (fy * inv_z).astype(F)
    j02 = -(((fx * xc).astype(F) * inv_z).astype(F))
    j12 = -(((fy * yc).astype(F) * inv_z).astype(F))
    # T = J Rc (2x3)
    T0 = [((j00 * r[0][k]).astype(F) + (j02 * r[2][k]).astype(F)).astype(F) for k in range(3)]
    T1 = [((j11 * r[1][k]).astype(F) + (j12 * r[2][k]).astype(F)).astype(F) for k in range(3)]

    # scale and rotation
    s = [exp32(lx), exp32(ly), exp32(lz)]
    qn2 = ((((qw * qw).astype(F) + (qx * qx).astype(F)).astype(F) + (qy * qy).astype(F)).astype(F)
           + (qz * qz).astype(F)).astype(F)
    ok &= qn2 > F(0.0)
    invn = (F(1.0) / np.sqrt(qn2).astype(F)).astype(F)
    w_, x_, y_, z_ = ((q * invn).astype(F) for q in (qw, qx, qy, qz))
    xx, yy, zz = (x_ * x_).astype(F), (y_ * y_).astype(F), (z_ * z_).astype(F)
    xy, xz, yz = (x_ * y_).astype(F), (x_ * z_).astype(F), (y_ * z_).astype(F)
    wx, wy, wz = (w_ * x_).astype(F), (w_ * y_).astype(F), (w_ * z_).astype(F)
    two, one = F(2.0), F(1.0)
    R = [[(one - (two * (yy + zz).astype(F)).astype(F)).astype(F),
          (two * (xy - wz).astype(F)).astype(F),
          (two * (xz + wy).astype(F)).astype(F)],
         [(two * (xy + wz).astype(F)).astype(F),
          (one - (two * (xx + zz).astype(F)).astype(F)).astype(F),
          (two * (yz - wx).astype(F)).astype(F)],
         [(two * (xz - wy).astype(F)).astype(F),
          (two * (yz + wx).astype(F)).astype(F),
          (one - (two * (xx + yy).astype(F)).astype(F)).astype(F)]]
    M = [[(R[i][j] * s[j]).astype(F) for j in range(3)] for i in range(3)]
    S = {}
    for (i, j) in ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)):
        S[i, j] = _dot3(M[i][0], M[i][1], M[i][2], M[j][0], M[j][1], M[j][2])
    S[1, 0], S[2, 0], S[2, 1] = S[0, 1], S[0, 2], S[1, 2]
    # U = T Sigma (2x3), Sigma' = U T^T (2x2)
    U0 = [_dot3(T0[0], T0[1], T0[2], S[0, k], S[1, k], S[2, k]) for k in range(3)]
    U1 = [_dot3(T1[0], T1[1], T1[2], S[0, k], S[1, k], S[2, k]) for k in range(3)]
    s00 = _dot3(U0[0], U0[1], U0[2], T0[0], T0[1], T0[2])
    s01 = _dot3(U0[0], U0[1], U0[2], T1[0], T1[1], T1[2])
    s11 = _dot3(U1[0], U1[1], U1[2], T1[0], T1[1], T1[2])
    a = (s00 + F(DILATION)).astype(F)
    b = s01
    c = (s11 + F(DILATION)).astype(F)
    det = ((a * c).astype(F) - (b * b).astype(F)).astype(F)
    ok &= det > F(0.0)
    inv_det = (F(1.0) / det).astype(F)
    ca = (c * inv_det).astype(F)
    cb = -((b * inv_det).astype(F))
    cc = (a * inv_det).astype(F)
    m = (F(0.5) * (a + c).astype(F)).astype(F)
    disc = np.maximum(F(LAMBDA_FLOOR), ((m * m).astype(F) - det).astype(F))
    lam = (m + np.sqrt(disc).astype(F)).astype(F)
    rad = np.ceil((F(3.0) * np.sqrt(lam).astype(F)).astype(F)).astype(F)

    # tile rectangle: tiles holding a pixel centre inside [u - r, u + r]^2
    lo_x = np.ceil((ux - rad).astype(F))
    hi_x = np.floor((ux + rad).astype(F))
    lo_y = np.ceil((uy - rad).astype(F))
    hi_y = np.floor((uy + rad).astype(F))
    ok &= (lo_x <= hi_x) & (lo_x <= F(W - 1)) & (hi_x >= F(0.0))
    ok &= (lo_y <= hi_y) & (lo_y <= F(H - 1)) & (hi_y >= F(0.0))

    # transfer-function cull (reading R5)
    if luts is not None:
        luts = np.asarray(luts, F)
        vis = np.zeros(n, bool)
        for lt in luts:
            A = tf_eval32(lt, v)[:, 3]
            o = (A * wt).astype(F)
            vis |= ~(o < F(ALPHA_MIN))
        ok &= vis

    ix0 = np.where(ok, np.maximum(lo_x, 0), 0).astype(np.int64)
    ix1 = np.where(ok, np.minimum(hi_x, W - 1), 0).astype(np.int64)
    iy0 = np.where(ok, np.maximum(lo_y, 0), 0).astype(np.int64)
    iy1 = np.where(ok, np.minimum(hi_y, H - 1), 0).astype(np.int64)
    rect = np.stack([ix0 // TILE, iy0 // TILE, ix1 // TILE + 1, iy1 // TILE + 1], 1)
    rect[~ok] = 0
    count = ((rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1])).astype(np.int64)
    geo = np.stack([ux, uy, tz, wt], 1).astype(F)
    aux = np.stack([ca, cb, cc, v], 1).astype(F)
    geo[~ok] = 0
    aux[~ok] = 0
    return {"geo": geo, "aux": aux, "count": count, "rect": rect, "valid": ok,
            "radius": np.where(ok, rad, 0).astype(F)}


# ============================================================================
# binning and depth sort (Sec. 3.3: the tile-based rasteriser)
# ============================================================================

def bin_sort(proj_views, cams):
    """Per-view tile lists.  For every visible Gaussian (in index order) and
    every tile of its rectangle (row-major), emit key = (view << (tb+32)) |
    (tile << 32) | bits(depth_f32) and value = view * N + index; sort keys
    stably.  Returns keys (uint64), vals (uint32), ranges (V, tiles, 2) and
    the tile-id bit width tb."""
    V = len(proj_views)
    tiles = cams[0].tiles_x * cams[0].tiles_y
    tb = max(1, int(math.ceil(math.log2(max(tiles, 2)))))
    keys, vals = [], []
    for vi, (p, cam) in enumerate(zip(proj_views, cams)):
        n = p["geo"].shape[0]
        dbits = p["geo"][:, 2].astype(F).view(np.uint32).astype(np.uint64)
        for gi in np.nonzero(p["count"] > 0)[0]:
            x0, y0, x1, y1 = p["rect"][gi]
            for ty in range(y0, y1):
                for tx in range(x0, x1):
                    tile = ty * cam.tiles_x + tx
                    keys.append((np.uint64(vi) << np.uint64(tb + 32))
                                | (np.uint64(tile) << np.uint64(32)) | dbits[gi])
                    vals.append(vi * n + gi)
    keys = np.array(keys, np.uint64)
    vals = np.array(vals, np.uint32)
    order = np.argsort(keys, kind="stable")
    keys, vals = keys[order], vals[order]
    ranges = np.zeros((V, tiles, 2), np.int64)
    if keys.size:
        vt = (keys >> np.uint64(32)).astype(np.int64)  # view * 2^tb + tile
        view = vt >> tb
        tile = vt & ((1 << tb) - 1)
        flat = view * tiles + tile
        starts = np.searchsorted(flat, np.arange(V * tiles), side="left")
        ends = np.searchsorted(flat, np.arange(V * tiles), side="right")
        ranges = np.stack([starts, ends], 1).reshape(V, tiles, 2)
        ranges[ranges[..., 0] == ranges[..., 1]] = 0
    return {"keys": keys, "vals": vals, "ranges": ranges, "tile_bits": tb}


# ============================================================================
# transfer function in float64 (reading R6)
# ============================================================================

def tf_eval64(lut, v):
    """Value and d/dv of the linear-interpolated table, float64."""
    lut = np.asarray(lut, np.float64)
    L = lut.shape[0]
    v = np.asarray(v, np.float64)
    vc = np.clip(v, 0.0, 1.0)
    p = vc * (L - 1)
    k = np.minimum(np.floor(p), L - 2).astype(np.int64)
    tau = p - k
    val = (1.0 - tau)[..., None] * lut[k] + tau[..., None] * lut[k + 1]
    inside = ((v >= 0.0) & (v <= 1.0)).astype(np.float64)
    slope = (L - 1) * (lut[k + 1] - lut[k]) * inside[..., None]
    return val, slope


# ============================================================================
# compositing, Eq. 1 (float64)
# ============================================================================

def _tile_pixels(cam, tile):
    tx, ty = tile % cam.tiles_x, tile // cam.tiles_x
    ys, xs = np.meshgrid(np.arange(16), np.arange(16), indexing="ij")
    px = (tx * 16 + xs).reshape(-1)
    py = (ty * 16 + ys).reshape(-1)
    keep = (px < cam.width) & (py < cam.height)
    return px[keep], py[keep]


def _flag_near(x, ref, rel):
    return np.abs(x / ref - 1.0) < rel


def _power_near_zero(qa, qc, qb, power):
    """The exponent -(qa + qc)/2 - qb is zero to within 1e-5 of the size of
    its terms: its sign (the skip of reading R7) is a rounding matter."""
    scale = np.abs(qa) + np.abs(qc) + 2 * np.abs(qb)
    return (np.abs(power) <= 1e-5 * scale) & (scale > 0)


def composite_tile(px, py, u, conic, v, w, luts, bg, frozen=None, record=False, shade=None):
    """Front-to-back blending (Eq. 1) of one tile's depth-sorted splats for
    the pixel centres (px, py) and every transfer function in `luts`.

    u (n,2), conic (n,3), v (n,), w (n,) are the tile's splats in list order;
    shade (n,2) optional Blinn-Phong factors (s_d, s_s): colour s_d C(v) + s_s.
    Returns dict(out (P,T,4), n_contrib (P,T), flag (P,T), stats, rec): rec
    holds per-splat (blend, clamped) masks when `record`.  With `frozen` (a
    previous rec) the threshold decisions are taken from it instead, which
    makes the result a smooth function of the splat parameters.
    """
    P = px.shape[0]
    nT = luts.shape[0]
    px = px.astype(np.float64)
    py = py.astype(np.float64)
    Tr = np.ones((P, nT))
    C = np.zeros((P, nT, 3))
    active = np.ones((P, nT), bool)
    last = np.zeros((P, nT), np.int64)
    flag = np.zeros((P, nT), bool)
    stats = {"visited": 0, "alpha_evals": 0, "blended": 0}
    rec = [] if record else None
    n = u.shape[0] if frozen is None else len(frozen)
    for i in range(n):
        if frozen is None and not active.any():
            break
        any_active = active.any(1)
        stats["visited"] += int(any_active.sum())
        dx = u[i, 0] - px
        dy = u[i, 1] - py
        a, b, c = conic[i]
        qa, qc, qb = a * dx * dx, c * dy * dy, b * dx * dy
        power = -0.5 * (qa + qc) - qb
        G = np.exp(power)
        vals = np.stack([tf_eval64(luts[t], v[i])[0] for t in range(nT)])  # (T,4)
        rgb = vals[:, :3]
        if shade is not None:
            rgb = shade[i, 0] * rgb + shade[i, 1]
        aw = vals[:, 3] * w[i]
        raw = G[:, None] * aw[None, :]
        alpha = np.minimum(ALPHA_MAX, raw)
        if frozen is None:
            ev = active & (power <= 0.0)[:, None]
            stats["alpha_evals"] += int(ev.sum())
            ok = ev & (alpha >= ALPHA_MIN)
            test = Tr * (1.0 - alpha)
            term = ok & (test < T_MIN)
            blend = ok & ~term
            clamped = blend & (raw > ALPHA_MAX)
            with np.errstate(divide="ignore", invalid="ignore"):
                near = (_flag_near(alpha, ALPHA_MIN, FLAG_ALPHA) | _flag_near(raw, ALPHA_MAX, FLAG_ALPHA)
                        | (ok & _flag_near(test, T_MIN, FLAG_T)))
                near |= _power_near_zero(qa, qc, qb, power)[:, None]
            flag |= active & near
            active &= ~term
        else:
            blend, clamped = frozen[i]
            alpha = np.where(clamped, ALPHA_MAX, raw)
            test = Tr * (1.0 - alpha)
        stats["blended"] += int(blend.sum())
        wgt = np.where(blend, alpha * Tr, 0.0)
        C += wgt[..., None] * rgb[None]
        Tr = np.where(blend, test, Tr)
        last = np.where(blend, i + 1, last)
        if record:
            rec.append((blend.copy(), clamped.copy()))
    out = np.concatenate([C + Tr[..., None] * np.asarray(bg, np.float64)[None, None],
                          Tr[..., None]], 2)
    return {"out": out, "n_contrib": last, "flag": flag, "stats": stats, "rec": rec}


def pixel_alternatives(x, y, u, conic, v, w, lut, bg, shade=None, limit=64):
    """Every outcome of Eq. 1 at the pixel centre (x, y) for one transfer
    function `lut` when each decision that lies inside a window of reading
    R12 may go either way: the skip of a positive exponent, the skip of
    alpha < 1/255 and the stop at T (1 - alpha) < 1e-4.  The splats (u,
    conic, v, w, shade) are the tile's list in order, as for composite_tile.

    Outside the windows each decision is the float64 one, so a pixel with no
    windowed decision has exactly one outcome, equal to composite_tile's.  A
    pair inside the window of the 0.99 clamp gives alpha = 0.99 to within
    1e-5 either way; it is not branched but marked (`clamp_near`), since its
    gradient depends on the side taken.

    Returns a list of dicts with out (4,) = (RGB + T bg, T_final), n_contrib,
    blend (n,) and clamped (n,) decisions and clamp_near; None when more than
    `limit` outcomes exist.
    """
    n = u.shape[0]
    lut = np.asarray(lut, np.float64)
    bg = np.asarray(bg, np.float64)
    dx = u[:, 0] - float(x)
    dy = u[:, 1] - float(y)
    a, b, c = conic[:, 0], conic[:, 1], conic[:, 2]
    qa, qc, qb = a * dx * dx, c * dy * dy, b * dx * dy
    power = -0.5 * (qa + qc) - qb
    pnear = _power_near_zero(qa, qc, qb, power)
    G = np.exp(power)
    vals = tf_eval64(lut, v)[0]  # (n, 4)
    rgb = vals[:, :3]
    if shade is not None:
        rgb = shade[:, :1] * rgb + shade[:, 1:2]
    raw = vals[:, 3] * w * G
    alpha = np.minimum(ALPHA_MAX, raw)
    with np.errstate(divide="ignore", invalid="ignore"):
        anear = _flag_near(alpha, ALPHA_MIN, FLAG_ALPHA)
        cnear = _flag_near(raw, ALPHA_MAX, FLAG_ALPHA)
    outs = []
    # depth-first over the windowed decisions; a state is the next list
    # position, T, the colour sum, n_contrib, the blended and clamped
    # positions so far and whether a clamp window was met
    stack = [(0, 1.0, np.zeros(3), 0, [], [], False)]
    while stack:
        i, T, C, last, bl, cl, cn = stack.pop()
        while i < n:
            evals = (False, True) if pnear[i] else (bool(power[i] <= 0.0),)
            if len(evals) == 2:
                stack.append((i + 1, T, C.copy(), last, list(bl), list(cl), cn))
                if len(stack) + len(outs) > limit:
                    return None
            if not evals[-1]:
                i += 1
                continue
            al = float(alpha[i])
            passes = (False, True) if anear[i] else (al >= ALPHA_MIN,)
            if len(passes) == 2:
                stack.append((i + 1, T, C.copy(), last, list(bl), list(cl), cn))
                if len(stack) + len(outs) > limit:
                    return None
            if not passes[-1]:
                i += 1
                continue
            test = T * (1.0 - al)
            if _flag_near(test, T_MIN, FLAG_T):
                # the side that stops here ends this outcome
                outs.append((T, C.copy(), last, list(bl), list(cl), cn))
                if len(stack) + len(outs) > limit:
                    return None
            elif test < T_MIN:
                break
            C = C + al * T * rgb[i]
            T = test
            last = i + 1
            bl.append(i)
            if raw[i] > ALPHA_MAX:
                cl.append(i)
            cn = cn or bool(cnear[i])
            i += 1
        outs.append((T, C, last, bl, cl, cn))
    res = []
    for T, C, last, bl, cl, cn in outs:
        blend = np.zeros(n, bool)
        blend[bl] = True
        clamped = np.zeros(n, bool)
        clamped[cl] = True
        res.append({"out": np.concatenate([C + T * bg, [T]]), "n_contrib": last,
                    "blend": blend, "clamped": clamped, "clamp_near": cn})
    return res


def flag_alternatives(proj_views, cams, bins, luts, bg, fwd, limit=64):
    """pixel_alternatives for every flagged (view, TF, y, x) of a forward
    result `fwd` (composite_fwd); returns {(view, tf, y, x): list or None}."""
    luts = np.asarray(luts, np.float64)
    res = {}
    cache = {}
    for vi, t, y, x in zip(*np.nonzero(fwd["flag"])):
        cam = cams[vi]
        tile = (y // TILE) * cam.tiles_x + x // TILE
        if (vi, tile) not in cache:
            proj = proj_views[vi]
            lo, hi = bins["ranges"][vi, tile]
            idx, u, conic, v, w = _tile_splats(proj, bins["vals"], lo, hi, proj["geo"].shape[0])
            cache[vi, tile] = (u, conic, v, w, _tile_shade(proj, idx))
        u, conic, v, w, sh = cache[vi, tile]
        res[int(vi), int(t), int(y), int(x)] = pixel_alternatives(x, y, u, conic, v, w, luts[t],
                                                                  bg, sh, limit)
    return res


def tile_pixel_index(cam, tile, x, y):
    """Position of pixel (x, y) in the pixel order of composite_tile (and of
    the recorded decisions) for `tile`."""
    px, py = _tile_pixels(cam, tile)
    return int(np.nonzero((px == x) & (py == y))[0][0])


def _tile_splats(proj, vals, lo, hi, n):
    idx = vals[lo:hi].astype(np.int64) % n
    geo = proj["geo"][idx].astype(np.float64)
    aux = proj["aux"][idx].astype(np.float64)
    return idx, geo[:, :2], aux[:, :3], aux[:, 3], geo[:, 3]


def _tile_shade(proj, idx):
    sh = proj.get("shade")
    return None if sh is None else np.asarray(sh, np.float64)[idx]


def composite_fwd(proj_views, cams, bins, luts, bg=(0.0, 0.0, 0.0), tiles=None,
                  record=False):
    """Render every view x transfer function.  Returns out (V,T,H,W,4),
    n_contrib (V,T,H,W), flag (V,T,H,W), stats and per-tile records.
    `tiles` restricts the work to a list of tile ids (crop mode)."""
    luts = np.asarray(luts, np.float64)
    V, nT = len(cams), luts.shape[0]
    H, W = cams[0].height, cams[0].width
    out = np.zeros((V, nT, H, W, 4))
    out[..., :3] = np.asarray(bg)
    out[..., 3] = 1.0
    nc = np.zeros((V, nT, H, W), np.int64)
    flag = np.zeros((V, nT, H, W), bool)
    stats = {"visited": 0, "alpha_evals": 0, "blended": 0}
    recs = {}
    ntiles = cams[0].tiles_x * cams[0].tiles_y
    for vi, (proj, cam) in enumerate(zip(proj_views, cams)):
        n = proj["geo"].shape[0]
        for tile in (range(ntiles) if tiles is None else tiles):
            lo, hi = bins["ranges"][vi, tile]
            px, py = _tile_pixels(cam, tile)
            idx, u, conic, v, w = _tile_splats(proj, bins["vals"], lo, hi, n)
            r = composite_tile(px, py, u, conic, v, w, luts, bg, record=record,
                               shade=_tile_shade(proj, idx))
            out[vi, :, py, px] = r["out"]
            nc[vi, :, py, px] = r["n_contrib"]
            flag[vi, :, py, px] = r["flag"]
            for k in stats:
                stats[k] += r["stats"][k]
            if record:
                recs[vi, tile] = r["rec"]
    return {"out": out, "n_contrib": nc, "flag": flag, "stats": stats, "rec": recs}


def composite_bwd_tile(px, py, u, conic, v, w, luts, bg, rec, dout, shade=None):
    """Gradients of one tile's blend w.r.t. each splat's screen mean, conic,
    scalar and weight (and shading factors), given the forward decisions
    `rec` and dL/d(out) `dout` (P,T,4).  Returns (n,9): du_x, du_y, da, db,
    dc, dv, dw, ds_d, ds_s (the last two zero without `shade`)."""
    P, nT = px.shape[0], luts.shape[0]
    n = len(rec)
    grad = np.zeros((u.shape[0], 9))
    if n == 0:
        return grad
    px = px.astype(np.float64)
    py = py.astype(np.float64)
    g = dout[..., :3]
    gT = dout[..., 3]
    bgv = np.asarray(bg, np.float64)
    steps = []
    Tr = np.ones((P, nT))
    for i in range(n):
        blend, clamped = rec[i]
        dx = u[i, 0] - px
        dy = u[i, 1] - py
        a, b, c = conic[i]
        power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
        G = np.exp(power)
        ev = [tf_eval64(luts[t], v[i]) for t in range(nT)]
        vals = np.stack([e[0] for e in ev])
        slopes = np.stack([e[1] for e in ev])
        aw = vals[:, 3] * w[i]
        raw = G[:, None] * aw[None]
        alpha = np.where(clamped, ALPHA_MAX, np.minimum(ALPHA_MAX, raw))
        sd, ss = (1.0, 0.0) if shade is None else (shade[i, 0], shade[i, 1])
        rgb = sd * vals[:, :3] + ss  # the blended colour
        cg = (g * rgb[None]).sum(-1)  # (P,T)
        steps.append((blend, clamped, dx, dy, power, G, vals, slopes, alpha, Tr.copy(), cg, sd))
        Tr = np.where(blend, Tr * (1.0 - alpha), Tr)
    T_final = Tr
    contrib = np.stack([np.where(s[0], s[10] * s[8] * s[9], 0.0) for s in steps])
    suffix = np.cumsum(contrib[::-1], 0)[::-1] - contrib
    K_end = T_final * ((g * bgv).sum(-1) + gT)
    for i, (blend, clamped, dx, dy, power, G, vals, slopes, alpha, Ti, cg, sd) in \
            enumerate(steps):
        if not blend.any():
            continue
        dalpha = np.where(blend, Ti * cg - (suffix[i] + K_end) / (1.0 - alpha), 0.0)
        wgt = np.where(blend, alpha * Ti, 0.0)  # dL/d(colour) = wgt * g
        free = blend & ~clamped
        A = vals[:, 3]
        daw = np.where(free, dalpha * G[:, None], 0.0)  # dL/d(A w)
        dG = np.where(free, dalpha * (A * w[i])[None], 0.0).sum(1)
        dv = ((sd * wgt[..., None] * g) * slopes[None, :, :3]).sum((1, 2)) \
            + (daw * w[i] * slopes[None, :, 3]).sum(1)
        dw = (daw * A[None]).sum(1)
        grad[i, 7] = (wgt[..., None] * g * vals[None, :, :3]).sum()
        grad[i, 8] = (wgt[..., None] * g).sum()
        dpow = dG * G
        a, b, c = conic[i]
        grad[i, 0] = (dpow * (-a * dx - b * dy)).sum()
        grad[i, 1] = (dpow * (-c * dy - b * dx)).sum()
        grad[i, 2] = (dpow * (-0.5 * dx * dx)).sum()
        grad[i, 3] = (dpow * (-dx * dy)).sum()
        grad[i, 4] = (dpow * (-0.5 * dy * dy)).sum()
        grad[i, 5] = dv.sum()
        grad[i, 6] = dw.sum()
    return grad


def composite_bwd(proj_views, cams, bins, luts, bg, fwd, dout, tiles=None):
    """Per-splat 2D gradients (V, N, 7) from dL/d(out) (V,T,H,W,4), using the
    forward decisions recorded in `fwd` (composite_fwd(..., record=True))."""
    luts = np.asarray(luts, np.float64)
    V = len(cams)
    n = proj_views[0]["geo"].shape[0]
    grad2d = np.zeros((V, n, 9))
    ntiles = cams[0].tiles_x * cams[0].tiles_y
    for vi, (proj, cam) in enumerate(zip(proj_views, cams)):
        for tile in (range(ntiles) if tiles is None else tiles):
            lo, hi = bins["ranges"][vi, tile]
            if hi <= lo:
                continue
            px, py = _tile_pixels(cam, tile)
            idx, u, conic, v, w = _tile_splats(proj, bins["vals"], lo, hi, n)
            d = np.transpose(dout[vi][:, py, px], (1, 0, 2))
            gt = composite_bwd_tile(px, py, u, conic, v, w, luts, bg, fwd["rec"][vi, tile], d,
                                    shade=_tile_shade(proj, idx))
            np.add.at(grad2d[vi], idx, gt)
    return grad2d


# ============================================================================
# projection in float64 and its backward (for the gradients, reading R9)
# ============================================================================

def _quat_rot64(q):
    qn = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = qn.T
    R = np.empty((q.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return qn, R


def project64(cam, mean, logscale, quat):
    """Screen mean u (N,2) and conic (N,3) in float64 (same maths as
    project32 without rounding), plus the intermediates the backward uses."""
    Rc = np.asarray(cam.world_to_cam, np.float64)[:, :3]
    tc = np.asarray(cam.world_to_cam, np.float64)[:, 3]
    t = mean @ Rc.T + tc
    tx, ty, tz = t.T
    xr, yr = tx / tz, ty / tz
    u = np.stack([cam.fx * xr + cam.cx, cam.fy * yr + cam.cy], 1)
    limx = FRUSTUM_SLACK * (0.5 * cam.width / cam.fx)
    limy = FRUSTUM_SLACK * (0.5 * cam.height / cam.fy)
    cx_ = np.abs(xr) <= limx
    cy_ = np.abs(yr) <= limy
    xc = np.clip(xr, -limx, limx)
    yc = np.clip(yr, -limy, limy)
    J = np.zeros((mean.shape[0], 2, 3))
    J[:, 0, 0] = cam.fx / tz
    J[:, 0, 2] = -cam.fx * xc / tz
    J[:, 1, 1] = cam.fy / tz
    J[:, 1, 2] = -cam.fy * yc / tz
    Tm = J @ Rc
    s = np.exp(logscale)
    qn, R = _quat_rot64(quat)
    Mm = R * s[:, None, :]
    Sig = Mm @ np.transpose(Mm, (0, 2, 1))
    Sp = Tm @ Sig @ np.transpose(Tm, (0, 2, 1))
    a = Sp[:, 0, 0] + DILATION
    b = Sp[:, 0, 1]
    c = Sp[:, 1, 1] + DILATION
    det = a * c - b * b
    conic = np.stack([c / det, -b / det, a / det], 1)
    return {"u": u, "conic": conic, "t": t, "Tm": Tm, "Sig": Sig, "Sp": np.stack([a, b, c], 1),
            "det": det, "s": s, "qn": qn, "R": R, "M": Mm, "Rc": Rc, "xc": xc, "yc": yc,
            "clip_x": cx_, "clip_y": cy_, "qnorm": np.linalg.norm(quat, axis=1)}


def project_bwd64(cam, fwd, d_u, d_conic):
    """Chain dL/du (N,2) and dL/d(conic a,b,c) (N,3) to the 3D mean,
    log-scale and quaternion (float64).  Returns (dmean, dlogscale, dquat)."""
    fx, fy = cam.fx, cam.fy
    t, Tm, Sig, Rc = fwd["t"], fwd["Tm"], fwd["Sig"], fwd["Rc"]
    tx, ty, tz = t.T
    a, b, c = fwd["Sp"].T
    det = fwd["det"]
    Q = np.zeros((t.shape[0], 2, 2))
    ca, cb, cc = (fwd["conic"][:, k] for k in range(3))
    Q[:, 0, 0], Q[:, 0, 1], Q[:, 1, 0], Q[:, 1, 1] = ca, cb, cb, cc
    GQ = np.zeros_like(Q)
    GQ[:, 0, 0] = d_conic[:, 0]
    GQ[:, 0, 1] = GQ[:, 1, 0] = 0.5 * d_conic[:, 1]
    GQ[:, 1, 1] = d_conic[:, 2]
    GS = -Q @ GQ @ Q                                 # dL/dSigma' (2x2 matrix)
    GSig = np.transpose(Tm, (0, 2, 1)) @ GS @ Tm     # dL/dSigma (3x3)
    GT = 2.0 * GS @ Tm @ Sig                         # dL/dT (2x3)
    GJ = GT @ Rc.T                                   # dL/dJ (2x3)
    dt = np.zeros_like(t)
    # u = f t_xy / t_z + c
    dt[:, 0] += d_u[:, 0] * fx / tz
    dt[:, 1] += d_u[:, 1] * fy / tz
    dt[:, 2] += -d_u[:, 0] * fx * tx / tz ** 2 - d_u[:, 1] * fy * ty / tz ** 2
    # J00 = fx/tz, J11 = fy/tz
    dt[:, 2] += -GJ[:, 0, 0] * fx / tz ** 2 - GJ[:, 1, 1] * fy / tz ** 2
    # J02 = -fx xc/tz with xc = tx/tz when unclamped
    cxm, cym = fwd["clip_x"], fwd["clip_y"]
    dt[:, 0] += np.where(cxm, -GJ[:, 0, 2] * fx / tz ** 2, 0.0)
    dt[:, 2] += np.where(cxm, GJ[:, 0, 2] * 2 * fx * tx / tz ** 3,
                         GJ[:, 0, 2] * fx * fwd["xc"] / tz ** 2)
    dt[:, 1] += np.where(cym, -GJ[:, 1, 2] * fy / tz ** 2, 0.0)
    dt[:, 2] += np.where(cym, GJ[:, 1, 2] * 2 * fy * ty / tz ** 3,
                         GJ[:, 1, 2] * fy * fwd["yc"] / tz ** 2)
    dmean = dt @ Rc
    # Sigma = M M^T, M = R diag(s)
    GM = 2.0 * GSig @ fwd["M"]
    s, R = fwd["s"], fwd["R"]
    GR = GM * s[:, None, :]
    ds = (GM * R).sum(1)
    dlogscale = ds * s
    w, x, y, z = fwd["qn"].T
    dqn = np.zeros((t.shape[0], 4))
    g = GR
    dqn[:, 0] = 2 * (-z * g[:, 0, 1] + y * g[:, 0, 2] + z * g[:, 1, 0] - x * g[:, 1, 2]
                     - y * g[:, 2, 0] + x * g[:, 2, 1])
    dqn[:, 1] = 2 * (y * g[:, 0, 1] + z * g[:, 0, 2] + y * g[:, 1, 0] - 2 * x * g[:, 1, 1]
                     - w * g[:, 1, 2] + z * g[:, 2, 0] + w * g[:, 2, 1] - 2 * x * g[:, 2, 2])
    dqn[:, 2] = 2 * (-2 * y * g[:, 0, 0] + x * g[:, 0, 1] + w * g[:, 0, 2] + x * g[:, 1, 0]
                     + z * g[:, 1, 2] - w * g[:, 2, 0] + z * g[:, 2, 1] - 2 * y * g[:, 2, 2])
    dqn[:, 3] = 2 * (-2 * z * g[:, 0, 0] - w * g[:, 0, 1] + x * g[:, 0, 2] + w * g[:, 1, 0]
                     - 2 * z * g[:, 1, 1] + y * g[:, 1, 2] + x * g[:, 2, 0] + y * g[:, 2, 1])
    qn = fwd["qn"]
    dquat = (dqn - qn * (qn * dqn).sum(1, keepdims=True)) / fwd["qnorm"][:, None]
    return dmean, dlogscale, dquat


def params_grad(cams, gs, proj_views, grad2d):
    """Sum over views of the chained gradients, packed like the inputs:
    (dmean, dv), (dlogscale, dw), dquat, each (N,4)."""
    n = gs.n
    gm = np.zeros((n, 4))
    gl = np.zeros((n, 4))
    gq = np.zeros((n, 4))
    mean = gs.mean_v[:, :3].astype(np.float64)
    ls = gs.logscale_w[:, :3].astype(np.float64)
    q = gs.quat.astype(np.float64)
    for vi, (cam, proj) in enumerate(zip(cams, proj_views)):
        ok = proj["valid"]
        if not ok.any():
            continue
        f = project64(cam, mean[ok], ls[ok], q[ok])
        g2 = grad2d[vi][ok]
        dm, dl, dq = project_bwd64(cam, f, g2[:, 0:2], g2[:, 2:5])
        gm[ok, :3] += dm
        gm[ok, 3] += g2[:, 5]
        gl[ok, :3] += dl
        gl[ok, 3] += g2[:, 6]
        gq[ok] += dq
    return gm, gl, gq


# ============================================================================
# loss (Sec. 4.2: the L1 part of the image loss)
# ============================================================================

def l1_loss(out, target):
    """Mean |out - target| over the RGB channels and dL/d(out) (zero on the
    transmittance channel; sign(0) = 0)."""
    d = np.asarray(out, np.float64)[..., :3] - np.asarray(target, np.float64)[..., :3]
    cnt = d.size
    grad = np.zeros(np.shape(out))
    grad[..., :3] = np.sign(d) / cnt
    return float(np.abs(d).sum() / cnt), grad


# ============================================================================
# whole path
# ============================================================================

def attach_shading(proj_views, cams, gs, lighting):
    """Adds the Blinn-Phong factors (s_d, s_s) of every view to its
    projection.  lighting: dict normal (N,3), ka, kd, ks, beta (N,), lights
    (V,3) unit world directions toward the light."""
    mean = gs.mean_v[:, :3].astype(np.float64)
    for vi, (p, cam) in enumerate(zip(proj_views, cams)):
        f = shade64(cam, lighting["lights"][vi], mean, np.asarray(lighting["normal"], np.float64),
                    *(np.asarray(lighting[k], np.float64) for k in ("ka", "kd", "ks", "beta")))
        p["shade"] = np.stack([f["s_d"], f["s_s"]], 1)
    return proj_views


def lighting_grad(cams, gs, lighting, proj_views, grad2d):
    """Chains the shading columns of grad2d (ds_d, ds_s) to the lighting
    parameters and the means, summed over views: returns dnormal (N,3),
    dka, dkd, dks, dbeta (N,), dmean (N,3)."""
    n = gs.n
    mean = gs.mean_v[:, :3].astype(np.float64)
    normal = np.asarray(lighting["normal"], np.float64)
    ka, kd, ks, beta = (np.asarray(lighting[k], np.float64) for k in ("ka", "kd", "ks", "beta"))
    acc = [np.zeros((n, 3)), np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n), np.zeros((n, 3))]
    for vi, (cam, proj) in enumerate(zip(cams, proj_views)):
        ok = proj["valid"]
        f = shade64(cam, lighting["lights"][vi], mean[ok], normal[ok], ka[ok], kd[ok], ks[ok],
                    beta[ok])
        parts = shade_bwd64(f, lighting["lights"][vi], ka[ok], kd[ok], ks[ok], beta[ok],
                            grad2d[vi][ok, 7], grad2d[vi][ok, 8])
        for a, p in zip(acc, parts):
            a[ok] += p
    return tuple(acc)


def render(cams, gs, luts, bg=(0.0, 0.0, 0.0), cull=True, tiles=None, record=False,
           lighting=None):
    """Project (per view), bin and sort, composite (Blinn-Phong shaded when
    `lighting` is given).  Returns (proj_views, bins, fwd)."""
    proj = [project32(c, gs, luts if cull else None) for c in cams]
    if lighting is not None:
        attach_shading(proj, cams, gs, lighting)
    bins = bin_sort(proj, cams)
    fwd = composite_fwd(proj, cams, bins, luts, bg, tiles=tiles, record=record)
    return proj, bins, fwd


def bruteforce_pixel(cam, proj, luts, bg, x, y):
    """Independent per-pixel evaluation: every visible Gaussian whose tile
    rectangle holds the pixel's tile, ordered by (float32 depth, index), blended
    one by one with scalar Python arithmetic (no keys, sorting network or
    ranges).  Returns (T, 4) and the list of n_contrib."""
    tx, ty = x // TILE, y // TILE
    cand = []
    for i in range(proj["geo"].shape[0]):
        if proj["count"][i] <= 0:
            continue
        x0, y0, x1, y1 = proj["rect"][i]
        if x0 <= tx < x1 and y0 <= ty < y1:
            cand.append((float(proj["geo"][i, 2]), i))
    cand.sort()
    res, ncs = [], []
    for lut in np.asarray(luts, np.float64):
        T, C, nc = 1.0, [0.0, 0.0, 0.0], 0
        L = lut.shape[0]
        for k, (_, i) in enumerate(cand):
            ux, uy = float(proj["geo"][i, 0]), float(proj["geo"][i, 1])
            a, b, c = (float(proj["aux"][i, j]) for j in range(3))
            v, w = float(proj["aux"][i, 3]), float(proj["geo"][i, 3])
            dx, dy = ux - x, uy - y
            power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
            if power > 0.0:
                continue
            pos = min(max(v, 0.0), 1.0) * (L - 1)
            j = min(int(math.floor(pos)), L - 2)
            fr = pos - j
            col = [(1 - fr) * lut[j, ch] + fr * lut[j + 1, ch] for ch in range(4)]
            alpha = min(ALPHA_MAX, col[3] * w * math.exp(power))
            if alpha < ALPHA_MIN:
                continue
            nt = T * (1.0 - alpha)
            if nt < T_MIN:
                break
            for ch in range(3):
                C[ch] += col[ch] * alpha * T
            T = nt
            nc = k + 1
        res.append([C[0] + T * bg[0], C[1] + T * bg[1], C[2] + T * bg[2], T])
        ncs.append(nc)
    return np.array(res), ncs


def render_frozen(cams, mean, logscale, quat, v, w, luts, bg, bins, recs, tiles, lighting=None):
    """The forward image as a smooth float64 function of the 3D parameters
    (and the lighting parameters): tile lists and every threshold decision
    are taken from an earlier recorded pass (`bins`, `recs`).  Used by the
    finite-difference pins."""
    luts = np.asarray(luts, np.float64)
    V, nT = len(cams), luts.shape[0]
    H, W = cams[0].height, cams[0].width
    n = mean.shape[0]
    out = np.zeros((V, nT, H, W, 4))
    out[..., :3] = np.asarray(bg)
    out[..., 3] = 1.0
    for vi, cam in enumerate(cams):
        f = project64(cam, mean, logscale, quat)
        shade = None
        if lighting is not None:
            s = shade64(cam, lighting["lights"][vi], mean, lighting["normal"], lighting["ka"],
                        lighting["kd"], lighting["ks"], lighting["beta"])
            shade = np.stack([s["s_d"], s["s_s"]], 1)
        for tile in tiles:
            lo, hi = bins["ranges"][vi, tile]
            px, py = _tile_pixels(cam, tile)
            idx = bins["vals"][lo:hi].astype(np.int64) % n
            r = composite_tile(px, py, f["u"][idx], f["conic"][idx], v[idx], w[idx], luts, bg,
                               frozen=recs[vi, tile], shade=None if shade is None else shade[idx])
            out[vi, :, py, px] = r["out"]
    return out


def tile_lists(proj, cam, tiles, view=0):
    """Lists of the given tiles by a direct rectangle test on every visible
    Gaussian, ordered by (float32 depth, index) -- no keys or global sort.
    Values are record indices view * n + i."""
    n = proj["geo"].shape[0]
    valid = proj["count"] > 0
    r = proj["rect"]
    depth = proj["geo"][:, 2]
    out = {}
    for tile in tiles:
        tx, ty = tile % cam.tiles_x, tile // cam.tiles_x
        m = valid & (r[:, 0] <= tx) & (tx < r[:, 2]) & (r[:, 1] <= ty) & (ty < r[:, 3])
        idx = np.nonzero(m)[0]
        idx = idx[np.lexsort((idx, depth[idx]))]
        out[tile] = idx + view * n
    return out


def bins_from_lists(lists_per_view, n_views, n_tiles):
    """A bins dict (vals, ranges) holding only the listed tiles."""
    vals, ranges, pos = [], np.zeros((n_views, n_tiles, 2), np.int64), 0
    for vi in range(n_views):
        for tile, lst in sorted(lists_per_view[vi].items()):
            ranges[vi, tile] = (pos, pos + len(lst)) if len(lst) else (0, 0)
            vals.append(np.asarray(lst, np.uint32))
            pos += len(lst)
    vals = np.concatenate(vals) if vals else np.zeros(0, np.uint32)
    return {"vals": vals, "ranges": ranges}


# ============================================================================
# Blinn-Phong shading (Eq. 2-3), float64
# ============================================================================
#
# Reading R16: the light is directional per view, `light` a unit world-space
# vector from the scene toward the light (the headlight of Sec. 4.2 / 5.1 is
# the camera's backward optical axis); v_i is the unit vector from the
# Gaussian's mean toward the camera centre; n_i is normalised.  Eq. 2-3 then
# read c_i = s_d C(v_i) + s_s white with
#     s_d = k^a + k^d |n.l|,  s_s = k^s |n.h|^beta if |n.l| > 0 else 0,
#     h = (v + l) / |v + l|.

def camera_centre(cam):
    w2c = np.asarray(cam.world_to_cam, np.float64)
    return -w2c[:, :3].T @ w2c[:, 3]


def headlight(cam):
    """Unit world direction toward a light on the camera's optical axis."""
    return -np.asarray(cam.world_to_cam, np.float64)[2, :3]


def shade64(cam, light, mean, normal, ka, kd, ks, beta):
    """(s_d, s_s) per Gaussian for one view, and the intermediates."""
    eye = camera_centre(cam)
    l = np.asarray(light, np.float64)
    vd = eye[None] - mean
    vlen = np.linalg.norm(vd, axis=1, keepdims=True)
    vh = vd / vlen
    nlen = np.linalg.norm(normal, axis=1, keepdims=True)
    nh_ = normal / nlen
    nl = nh_ @ l
    hv = vh + l[None]
    hlen = np.linalg.norm(hv, axis=1, keepdims=True)
    h = hv / hlen
    ndh = (nh_ * h).sum(1)
    s_d = ka + kd * np.abs(nl)
    lit = np.abs(nl) > 0
    with np.errstate(divide="ignore", invalid="ignore"):
        s_s = np.where(lit, ks * np.abs(ndh) ** beta, 0.0)
    return {"s_d": s_d, "s_s": s_s, "nl": nl, "ndh": ndh, "n_hat": nh_, "nlen": nlen[:, 0],
            "v_hat": vh, "vlen": vlen[:, 0], "h": h, "hlen": hlen[:, 0], "lit": lit}


def shade_bwd64(f, light, ka, kd, ks, beta, d_sd, d_ss):
    """Chains dL/ds_d and dL/ds_s to (dnormal (N,3), dka, dkd, dks, dbeta,
    dmean (N,3)); derivatives of |.| use sign (0 at 0)."""
    l = np.asarray(light, np.float64)
    nl, ndh = f["nl"], f["ndh"]
    sgn_l = np.sign(nl)
    sgn_h = np.sign(ndh)
    a = np.abs(ndh)
    with np.errstate(divide="ignore", invalid="ignore"):
        pw = np.where(f["lit"] & (a > 0), a ** beta, 0.0)
        dpw_da = np.where(f["lit"] & (a > 0), beta * a ** (beta - 1.0), 0.0)
        dpw_db = np.where(f["lit"] & (a > 0), pw * np.log(np.where(a > 0, a, 1.0)), 0.0)
    dka = d_sd
    dkd = d_sd * np.abs(nl)
    dks = d_ss * pw
    dbeta = d_ss * ks * dpw_db
    g_nl = d_sd * kd * sgn_l                       # dL/d(n_hat . l)
    g_ndh = d_ss * ks * dpw_da * sgn_h             # dL/d(n_hat . h)
    g_nhat = g_nl[:, None] * l[None] + g_ndh[:, None] * f["h"]
    nh_ = f["n_hat"]
    dnormal = (g_nhat - nh_ * (nh_ * g_nhat).sum(1, keepdims=True)) / f["nlen"][:, None]
    # h = (v_hat + l) / |v_hat + l|, v_hat = (eye - mean) / |eye - mean|
    g_h = g_ndh[:, None] * nh_
    h = f["h"]
    g_hv = (g_h - h * (h * g_h).sum(1, keepdims=True)) / f["hlen"][:, None]
    vh = f["v_hat"]
    g_vd = (g_hv - vh * (vh * g_hv).sum(1, keepdims=True)) / f["vlen"][:, None]
    dmean = -g_vd
    return dnormal, dka, dkd, dks, dbeta, dmean
