// Projection of VEG Gaussians to screen space and its backward pass.
//
// Forward (Sec. 3.3): Sigma = R S S^T R^T from the quaternion and the
// per-axis scale, EWA projection Sigma' = J W Sigma W^T J^T (Zwicker et al.),
// conic = Sigma'^-1, tile rectangle from a 3-sigma radius, and the optional
// transfer-function cull (TF applied first; Gaussians mapped to alpha below
// 1/255 are dropped).  Every binning-critical value is computed with
// explicitly rounded float32 operations in a fixed order (no contraction).
//
// Backward (Sec. 3.3, manual gradients): screen-space gradients of
// (u, conic, v, w) are chained to the mean, log-scale and quaternion and
// summed over views; one thread owns one Gaussian, so no atomics.
#include "veg_internal.cuh"

namespace veg {

namespace {

struct Proj {
  float tx, ty, tz, inv_z;
  float ux, uy;
  float xr, yr;
  bool clip_x, clip_y;  // true when the Jacobian ratio is clamped
  float T0[3], T1[3];   // T = J W (2x3)
  float s[3];
  float qw, qx, qy, qz;  // normalised quaternion
  float invn;            // 1 / |q|
  float R[3][3];
  float M[3][3];
  float S[3][3];
  float a, b, c;  // Sigma' + 0.3 I
  float det;
  float ca, cb, cc;
};

// Float32 projection in the fixed operation order.  Returns false when the
// Gaussian is culled by the near plane, a zero quaternion or det <= 0.
__device__ __forceinline__ bool project_one(const CamParam& cp, float4 mv, float4 lw, float4 q,
                                            Proj& P) {
  const float* r = cp.r;
  P.tx = add(dot3(r[0], r[1], r[2], mv.x, mv.y, mv.z), cp.t[0]);
  P.ty = add(dot3(r[3], r[4], r[5], mv.x, mv.y, mv.z), cp.t[1]);
  P.tz = add(dot3(r[6], r[7], r[8], mv.x, mv.y, mv.z), cp.t[2]);
  bool ok = P.tz > cp.near_plane;
  P.inv_z = dv(1.0f, P.tz);
  P.xr = mul(P.tx, P.inv_z);
  P.yr = mul(P.ty, P.inv_z);
  P.ux = add(mul(cp.fx, P.xr), cp.cx);
  P.uy = add(mul(cp.fy, P.yr), cp.cy);
  float limx = mul(kFrustumSlack, dv(mul(0.5f, (float)cp.width), cp.fx));
  float limy = mul(kFrustumSlack, dv(mul(0.5f, (float)cp.height), cp.fy));
  float xc = fminf(fmaxf(P.xr, -limx), limx);
  float yc = fminf(fmaxf(P.yr, -limy), limy);
  P.clip_x = !(fabsf(P.xr) <= limx);
  P.clip_y = !(fabsf(P.yr) <= limy);
  float j00 = mul(cp.fx, P.inv_z);
  float j11 = mul(cp.fy, P.inv_z);
  float j02 = -mul(mul(cp.fx, xc), P.inv_z);
  float j12 = -mul(mul(cp.fy, yc), P.inv_z);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    P.T0[k] = add(mul(j00, r[k]), mul(j02, r[6 + k]));
    P.T1[k] = add(mul(j11, r[3 + k]), mul(j12, r[6 + k]));
  }
  P.s[0] = exp_cw(lw.x);
  P.s[1] = exp_cw(lw.y);
  P.s[2] = exp_cw(lw.z);
  float qn2 = add(add(add(mul(q.x, q.x), mul(q.y, q.y)), mul(q.z, q.z)), mul(q.w, q.w));
  ok = ok && (qn2 > 0.0f);
  P.invn = dv(1.0f, sqrt_rn(qn2));
  float w = mul(q.x, P.invn), x = mul(q.y, P.invn), y = mul(q.z, P.invn), z = mul(q.w, P.invn);
  P.qw = w;
  P.qx = x;
  P.qy = y;
  P.qz = z;
  float xx = mul(x, x), yy = mul(y, y), zz = mul(z, z);
  float xy = mul(x, y), xz = mul(x, z), yz = mul(y, z);
  float wx = mul(w, x), wy = mul(w, y), wz = mul(w, z);
  P.R[0][0] = sub(1.0f, mul(2.0f, add(yy, zz)));
  P.R[0][1] = mul(2.0f, sub(xy, wz));
  P.R[0][2] = mul(2.0f, add(xz, wy));
  P.R[1][0] = mul(2.0f, add(xy, wz));
  P.R[1][1] = sub(1.0f, mul(2.0f, add(xx, zz)));
  P.R[1][2] = mul(2.0f, sub(yz, wx));
  P.R[2][0] = mul(2.0f, sub(xz, wy));
  P.R[2][1] = mul(2.0f, add(yz, wx));
  P.R[2][2] = sub(1.0f, mul(2.0f, add(xx, yy)));
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) P.M[i][j] = mul(P.R[i][j], P.s[j]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      P.S[i][j] = dot3(P.M[i][0], P.M[i][1], P.M[i][2], P.M[j][0], P.M[j][1], P.M[j][2]);
      P.S[j][i] = P.S[i][j];
    }
  float U0[3], U1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    U0[k] = dot3(P.T0[0], P.T0[1], P.T0[2], P.S[0][k], P.S[1][k], P.S[2][k]);
    U1[k] = dot3(P.T1[0], P.T1[1], P.T1[2], P.S[0][k], P.S[1][k], P.S[2][k]);
  }
  float s00 = dot3(U0[0], U0[1], U0[2], P.T0[0], P.T0[1], P.T0[2]);
  float s01 = dot3(U0[0], U0[1], U0[2], P.T1[0], P.T1[1], P.T1[2]);
  float s11 = dot3(U1[0], U1[1], U1[2], P.T1[0], P.T1[1], P.T1[2]);
  P.a = add(s00, kDilation);
  P.b = s01;
  P.c = add(s11, kDilation);
  P.det = sub(mul(P.a, P.c), mul(P.b, P.b));
  ok = ok && (P.det > 0.0f);
  float inv_det = dv(1.0f, P.det);
  P.ca = mul(P.c, inv_det);
  P.cb = -mul(P.b, inv_det);
  P.cc = mul(P.a, inv_det);
  return ok;
}

// Record o of `view`: the projection of Gaussian (mv, lw, q).
__device__ __forceinline__ void project_record(const CamParam& cp, int view, float4 mv, float4 lw,
                                               float4 q, int64_t o,
                                               const float4* __restrict__ cull_lut, int lut_size,
                                               int n_tf, const int32_t* __restrict__ view_tf,
                                               float4* __restrict__ geo, float4* __restrict__ aux,
                                               int32_t* __restrict__ tiles,
                                               short4* __restrict__ rect) {
  Proj P;
  bool ok = project_one(cp, mv, lw, q, P);
  // radius from the larger eigenvalue of Sigma'
  float m = mul(0.5f, add(P.a, P.c));
  float disc = fmaxf(kLambdaFloor, sub(mul(m, m), P.det));
  float lam = add(m, sqrt_rn(disc));
  float rad = ceilf(mul(3.0f, sqrt_rn(lam)));
  float lo_x = ceilf(sub(P.ux, rad)), hi_x = floorf(add(P.ux, rad));
  float lo_y = ceilf(sub(P.uy, rad)), hi_y = floorf(add(P.uy, rad));
  ok = ok && (lo_x <= hi_x) && (lo_x <= (float)(cp.width - 1)) && (hi_x >= 0.0f);
  ok = ok && (lo_y <= hi_y) && (lo_y <= (float)(cp.height - 1)) && (hi_y >= 0.0f);
  if (ok && cull_lut != nullptr) {
    TfPos tp = tf_pos(mv.w, lut_size);
    bool vis = false;
    int t_lo = 0, t_hi = n_tf;
    if (view_tf != nullptr) {  // this view is composited with one table only
      t_lo = view_tf[view];
      t_hi = t_lo + 1;
      if (t_lo < 0 || t_lo >= n_tf) t_lo = t_hi = 0;  // transparent table: cull
    }
    for (int t = t_lo; t < t_hi && !vis; ++t) {
      const float4* L = cull_lut + (int64_t)t * lut_size;
      float A = lerp_rn(__ldg(&L[tp.k].w), __ldg(&L[tp.k + 1].w), tp);
      vis = !(mul(A, lw.w) < kAlphaMin);
    }
    ok = vis;
  }
  if (!ok) {
    geo[o] = make_float4(0.f, 0.f, 0.f, 0.f);
    aux[o] = make_float4(0.f, 0.f, 0.f, 0.f);
    tiles[o] = 0;
    rect[o] = make_short4(0, 0, 0, 0);
    return;
  }
  int ix0 = (int)fmaxf(lo_x, 0.0f), ix1 = (int)fminf(hi_x, (float)(cp.width - 1));
  int iy0 = (int)fmaxf(lo_y, 0.0f), iy1 = (int)fminf(hi_y, (float)(cp.height - 1));
  short x0 = (short)(ix0 >> 4), x1 = (short)((ix1 >> 4) + 1);
  short y0 = (short)(iy0 >> 4), y1 = (short)((iy1 >> 4) + 1);
  geo[o] = make_float4(P.ux, P.uy, P.tz, lw.w);
  aux[o] = make_float4(P.ca, P.cb, P.cc, mv.w);
  tiles[o] = (int32_t)(x1 - x0) * (int32_t)(y1 - y0);
  rect[o] = make_short4(x0, y0, x1, y1);
}

__global__ void __launch_bounds__(256)
    project_fwd_kernel(CamSet cams, const float4* __restrict__ mean_v,
                       const float4* __restrict__ logscale_w, const float4* __restrict__ quat,
                       int64_t n, const float4* __restrict__ cull_lut, int lut_size, int n_tf,
                       const int32_t* __restrict__ view_tf, float4* __restrict__ geo,
                       float4* __restrict__ aux,
                       int32_t* __restrict__ tiles, short4* __restrict__ rect) {
  pdl_enter();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int view = blockIdx.y;
  project_record(cams.c[view], view, mean_v[i], logscale_w[i], quat[i], (int64_t)view * n + i,
                 cull_lut, lut_size, n_tf, view_tf, geo, aux, tiles, rect);
}

// Each view its own model: view v projects models.n[v] Gaussians into its
// records [v n, v n + models.n[v]); its records up to (v + 1) n only get
// tiles_touched = 0 (the binning reads nothing else of a record that
// touches no tile).
__global__ void __launch_bounds__(256)
    project_views_kernel(CamSet cams, const __grid_constant__ ViewModels models, int64_t n,
                         const float4* __restrict__ cull_lut, int lut_size, int n_tf,
                         const int32_t* __restrict__ view_tf, float4* __restrict__ geo,
                         float4* __restrict__ aux, int32_t* __restrict__ tiles,
                         short4* __restrict__ rect) {
  pdl_enter();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int view = blockIdx.y;
  const int64_t o = (int64_t)view * n + i;
  if (i >= models.n[view]) {
    tiles[o] = 0;
    return;
  }
  project_record(cams.c[view], view, models.mean_v[view][i], models.logscale_w[view][i],
                 models.quat[view][i], o, cull_lut, lut_size, n_tf, view_tf, geo, aux, tiles,
                 rect);
}

// dL/d(u, conic) of one view chained to the 3D parameters (accumulated).
__device__ __forceinline__ void project_bwd_one(const CamParam& cp, const Proj& P, float4 g0,
                                                float4 g1, float dm[3], float dl[3],
                                                float dq[4]) {
  const float* r = cp.r;
  const float fx = cp.fx, fy = cp.fy;
  // dL/dSigma' = -Q GQ Q, Q = [[ca, cb], [cb, cc]], GQ = [[da, db/2], [db/2, dc]]
  float da = g0.z, db = 0.5f * g0.w, dc = g1.x;
  float q00 = P.ca, q01 = P.cb, q11 = P.cc;
  float m00 = da * q00 + db * q01, m01 = da * q01 + db * q11;
  float m10 = db * q00 + dc * q01, m11 = db * q01 + dc * q11;
  float gs00 = -(q00 * m00 + q01 * m10);
  float gs01 = -(q00 * m01 + q01 * m11);
  float gs11 = -(q01 * m01 + q11 * m11);
  // dL/dSigma = T^T GS T
  float GT0[3], GT1[3];  // GS T (2x3)
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    GT0[k] = gs00 * P.T0[k] + gs01 * P.T1[k];
    GT1[k] = gs01 * P.T0[k] + gs11 * P.T1[k];
  }
  float GSig[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) GSig[i][j] = P.T0[i] * GT0[j] + P.T1[i] * GT1[j];
  // dL/dT = 2 GS T Sigma ; dL/dJ = dL/dT W^T (only J00, J02, J11, J12 vary)
  float GTm0[3], GTm1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    GTm0[k] = 2.0f * (GT0[0] * P.S[0][k] + GT0[1] * P.S[1][k] + GT0[2] * P.S[2][k]);
    GTm1[k] = 2.0f * (GT1[0] * P.S[0][k] + GT1[1] * P.S[1][k] + GT1[2] * P.S[2][k]);
  }
  float gj00 = GTm0[0] * r[0] + GTm0[1] * r[1] + GTm0[2] * r[2];
  float gj02 = GTm0[0] * r[6] + GTm0[1] * r[7] + GTm0[2] * r[8];
  float gj11 = GTm1[0] * r[3] + GTm1[1] * r[4] + GTm1[2] * r[5];
  float gj12 = GTm1[0] * r[6] + GTm1[1] * r[7] + GTm1[2] * r[8];
  const float iz = P.inv_z, iz2 = iz * iz, iz3 = iz2 * iz;
  float dtx = g0.x * fx * iz;
  float dty = g0.y * fy * iz;
  float dtz = -(g0.x * fx * P.tx + g0.y * fy * P.ty) * iz2;
  dtz += -(gj00 * fx + gj11 * fy) * iz2;
  if (!P.clip_x) {
    dtx += -gj02 * fx * iz2;
    dtz += gj02 * 2.0f * fx * P.tx * iz3;
  } else {
    float lim = kFrustumSlack * (0.5f * cp.width / fx);
    dtz += gj02 * fx * fminf(fmaxf(P.xr, -lim), lim) * iz2;
  }
  if (!P.clip_y) {
    dty += -gj12 * fy * iz2;
    dtz += gj12 * 2.0f * fy * P.ty * iz3;
  } else {
    float lim = kFrustumSlack * (0.5f * cp.height / fy);
    dtz += gj12 * fy * fminf(fmaxf(P.yr, -lim), lim) * iz2;
  }
  dm[0] += r[0] * dtx + r[3] * dty + r[6] * dtz;
  dm[1] += r[1] * dtx + r[4] * dty + r[7] * dtz;
  dm[2] += r[2] * dtx + r[5] * dty + r[8] * dtz;
  // Sigma = M M^T, M = R diag(s)
  float GR[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float gm = 2.0f * (GSig[i][0] * P.M[0][j] + GSig[i][1] * P.M[1][j] + GSig[i][2] * P.M[2][j]);
      GR[i][j] = gm * P.s[j];
      dl[j] += gm * P.R[i][j] * P.s[j];
    }
  const float w = P.qw, x = P.qx, y = P.qy, z = P.qz;
  float dw = 2.0f * (-z * GR[0][1] + y * GR[0][2] + z * GR[1][0] - x * GR[1][2] - y * GR[2][0] +
                     x * GR[2][1]);
  float dx = 2.0f * (y * GR[0][1] + z * GR[0][2] + y * GR[1][0] - 2.0f * x * GR[1][1] -
                     w * GR[1][2] + z * GR[2][0] + w * GR[2][1] - 2.0f * x * GR[2][2]);
  float dy = 2.0f * (-2.0f * y * GR[0][0] + x * GR[0][1] + w * GR[0][2] + x * GR[1][0] +
                     z * GR[1][2] - w * GR[2][0] + z * GR[2][1] - 2.0f * y * GR[2][2]);
  float dz = 2.0f * (-2.0f * z * GR[0][0] - w * GR[0][1] + x * GR[0][2] + w * GR[1][0] -
                     2.0f * z * GR[1][1] + y * GR[1][2] + x * GR[2][0] + y * GR[2][1]);
  float dot = w * dw + x * dx + y * dy + z * dz;
  dq[0] += (dw - w * dot) * P.invn;
  dq[1] += (dx - x * dot) * P.invn;
  dq[2] += (dy - y * dot) * P.invn;
  dq[3] += (dz - z * dot) * P.invn;
}

// Six CTAs per SM (80 registers): the per-Gaussian chain is latency-bound,
// and the extra resident warps outweigh a few spilled registers (36% faster
// than one CTA's 116 registers on the training step).
__global__ void __launch_bounds__(128, 6)
    project_bwd_kernel(CamSet cams, int n_views, const float4* __restrict__ mean_v,
                       const float4* __restrict__ logscale_w, const float4* __restrict__ quat,
                       int64_t n, int64_t first, int64_t end, const int32_t* __restrict__ tiles,
                       const float4* __restrict__ grad2d, float4* __restrict__ grad_mean_v,
                       float4* __restrict__ grad_logscale_w, float4* __restrict__ grad_quat) {
  pdl_enter();
  int64_t i = first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= end) return;
  float4 mv = mean_v[i], lw = logscale_w[i], q = quat[i];
  float dm[3] = {0.f, 0.f, 0.f}, dl[3] = {0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f};
  float dvv = 0.f, dww = 0.f;
  bool any = false;
  for (int view = 0; view < n_views; ++view) {
    int64_t o = (int64_t)view * n + i;
    if (tiles[o] == 0) continue;
    float4 g0 = grad2d[2 * o], g1 = grad2d[2 * o + 1];
    if (g0.x == 0.f && g0.y == 0.f && g0.z == 0.f && g0.w == 0.f && g1.x == 0.f && g1.y == 0.f &&
        g1.z == 0.f)
      continue;
    any = true;
    Proj P;
    project_one(cams.c[view], mv, lw, q, P);
    project_bwd_one(cams.c[view], P, g0, g1, dm, dl, dq);
    dvv += g1.y;
    dww += g1.z;
  }
  if (!any) return;
  // add into the gradients with vector reductions instead of a load and a
  // store: the thread retires without waiting for a read
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(grad_mean_v + i), "f"(dm[0]),
               "f"(dm[1]), "f"(dm[2]), "f"(dvv) : "memory");
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(grad_logscale_w + i),
               "f"(dl[0]), "f"(dl[1]), "f"(dl[2]), "f"(dww) : "memory");
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(grad_quat + i), "f"(dq[0]),
               "f"(dq[1]), "f"(dq[2]), "f"(dq[3]) : "memory");
}

}  // namespace

veg_status project_launch(const CamSet& cs, int n_views, veg_gaussians g, const veg_tf* cull_tf,
                          float4* geo, float4* aux, int32_t* tiles, short4* rect,
                          cudaStream_t stream) {
  if (g.n == 0) return VEG_OK;
  dim3 grid((unsigned)((g.n + 255) / 256), (unsigned)n_views);
  const float4* lut = cull_tf ? reinterpret_cast<const float4*>(cull_tf->lut) : nullptr;
  launch_k(project_fwd_kernel, grid, 256, 0, stream, 
      cs, reinterpret_cast<const float4*>(g.mean_v), reinterpret_cast<const float4*>(g.logscale_w),
      reinterpret_cast<const float4*>(g.quat), g.n, lut, cull_tf ? cull_tf->lut_size : 0,
      cull_tf ? cull_tf->n_tf : 0, cull_tf ? cull_tf->view_tf : nullptr, geo, aux, tiles, rect);
  count_launch();
  return launch_status();
}

veg_status project_views_launch(const CamSet& cs, int n_views, const ViewModels& models,
                                int64_t n, const veg_tf* cull_tf, float4* geo, float4* aux,
                                int32_t* tiles, short4* rect, cudaStream_t stream) {
  if (n == 0) return VEG_OK;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)n_views);
  const float4* lut = cull_tf ? reinterpret_cast<const float4*>(cull_tf->lut) : nullptr;
  launch_k(project_views_kernel, grid, 256, 0, stream, cs, models, n, lut,
           cull_tf ? cull_tf->lut_size : 0, cull_tf ? cull_tf->n_tf : 0,
           cull_tf ? cull_tf->view_tf : nullptr, geo, aux, tiles, rect);
  count_launch();
  return launch_status();
}

veg_status project_bwd_launch(const CamSet& cs, int n_views, veg_gaussians g,
                              const int32_t* tiles, const float4* grad2d, float4* gm, float4* gl,
                              float4* gq, cudaStream_t stream, int64_t first, int64_t count) {
  if (count < 0) count = g.n - first;
  if (count == 0) return VEG_OK;
  dim3 grid((unsigned)((count + 127) / 128));
  launch_k(project_bwd_kernel, grid, 128, 0, stream, 
      cs, n_views, reinterpret_cast<const float4*>(g.mean_v),
      reinterpret_cast<const float4*>(g.logscale_w), reinterpret_cast<const float4*>(g.quat), g.n,
      first, first + count, tiles, grad2d, gm, gl, gq);
  count_launch();
  return launch_status();
}

}  // namespace veg

extern "C" veg_status veg_project(const veg_camera* cams, int32_t n_views, veg_gaussians g,
                                  const veg_tf* cull_tf, float* splat_geo, float* splat_aux,
                                  int32_t* tiles_touched, int16_t* rect, cudaStream_t stream) {
  using namespace veg;
  veg_status st = check_cameras(cams, n_views);
  if (st != VEG_OK) return st;
  if (g.n < 0 || (g.n > 0 && (!g.mean_v || !g.logscale_w || !g.quat || !splat_geo ||
                              !splat_aux || !tiles_touched || !rect)))
    return VEG_ERR_INVALID_ARGUMENT;
  if (g.n > ((int64_t)1 << 31) / n_views) return VEG_ERR_INVALID_ARGUMENT;
  if (!aligned16(g.mean_v) || !aligned16(g.logscale_w) || !aligned16(g.quat) ||
      !aligned16(splat_geo) || !aligned16(splat_aux) || (reinterpret_cast<uintptr_t>(rect) & 7))
    return VEG_ERR_INVALID_ARGUMENT;
  if (cull_tf && (!cull_tf->lut || cull_tf->lut_size < 2 || cull_tf->n_tf < 1 ||
                  !aligned16(cull_tf->lut)))
    return VEG_ERR_INVALID_ARGUMENT;
  CamSet cs;
  fill_camset(cams, n_views, &cs);
  return project_launch(cs, n_views, g, cull_tf, reinterpret_cast<float4*>(splat_geo),
                        reinterpret_cast<float4*>(splat_aux), tiles_touched,
                        reinterpret_cast<short4*>(rect), stream);
}

extern "C" veg_status veg_project_views(const veg_camera* cams, int32_t n_views,
                                        const veg_gaussians* models, int64_t n,
                                        const veg_tf* cull_tf, float* splat_geo,
                                        float* splat_aux, int32_t* tiles_touched, int16_t* rect,
                                        cudaStream_t stream) {
  using namespace veg;
  veg_status st = check_cameras(cams, n_views);
  if (st != VEG_OK) return st;
  if (!models || n < 0 || n > ((int64_t)1 << 31) / n_views) return VEG_ERR_INVALID_ARGUMENT;
  if (n > 0 && (!splat_geo || !splat_aux || !tiles_touched || !rect))
    return VEG_ERR_INVALID_ARGUMENT;
  if (!aligned16(splat_geo) || !aligned16(splat_aux) || (reinterpret_cast<uintptr_t>(rect) & 7))
    return VEG_ERR_INVALID_ARGUMENT;
  ViewModels vm;
  for (int v = 0; v < n_views; ++v) {
    const veg_gaussians& g = models[v];
    if (g.n < 0 || g.n > n) return VEG_ERR_INVALID_ARGUMENT;
    if (g.n > 0 && (!g.mean_v || !g.logscale_w || !g.quat || !aligned16(g.mean_v) ||
                    !aligned16(g.logscale_w) || !aligned16(g.quat)))
      return VEG_ERR_INVALID_ARGUMENT;
    vm.mean_v[v] = reinterpret_cast<const float4*>(g.mean_v);
    vm.logscale_w[v] = reinterpret_cast<const float4*>(g.logscale_w);
    vm.quat[v] = reinterpret_cast<const float4*>(g.quat);
    vm.n[v] = g.n;
  }
  if (cull_tf && (!cull_tf->lut || cull_tf->lut_size < 2 || cull_tf->n_tf < 1 ||
                  !aligned16(cull_tf->lut)))
    return VEG_ERR_INVALID_ARGUMENT;
  CamSet cs;
  fill_camset(cams, n_views, &cs);
  return project_views_launch(cs, n_views, vm, n, cull_tf, reinterpret_cast<float4*>(splat_geo),
                              reinterpret_cast<float4*>(splat_aux), tiles_touched,
                              reinterpret_cast<short4*>(rect), stream);
}
