// Blinn-Phong shading of VEG Gaussians (Eq. 2-3) and its backward pass.
//
// Per view and Gaussian the colour of Eq. 2 is c = s_d C(v) + s_s white with
//   s_d = k^a + k^d |n.l|,   s_s = k^s |n.h|^beta if |n.l| > 0 else 0,
// n the normalised normal, l the view's unit light direction (toward the
// light; a headlight lies on the camera's backward optical axis), h the unit
// half vector of l and the unit direction from the Gaussian to the camera.
// The factors depend on the view but not on the transfer function, so they
// are computed once per (view, Gaussian) and read by the compositor.
#include <cmath>

#include "veg_internal.cuh"

namespace veg {

namespace {

struct LightSet {
  float l[VEG_MAX_VIEWS][3];    // unit light direction
  float eye[VEG_MAX_VIEWS][3];  // camera centre, world
};

struct ShadeTerms {
  float nh[3], nlen;  // normalised normal, |n|
  float vh[3], vlen;  // unit direction to the camera, distance
  float h[3], hlen;   // unit half vector, |v + l|
  float nl, ndh;      // n.l, n.h
  float sd, ss;
};

__device__ __forceinline__ ShadeTerms shade_terms(const float l[3], const float eye[3], float3 mu,
                                                  float4 nb, float4 k) {
  ShadeTerms S;
  float vx = eye[0] - mu.x, vy = eye[1] - mu.y, vz = eye[2] - mu.z;
  S.vlen = sqrtf(vx * vx + vy * vy + vz * vz);
  const float iv = S.vlen > 0.f ? 1.0f / S.vlen : 0.f;
  S.vh[0] = vx * iv;
  S.vh[1] = vy * iv;
  S.vh[2] = vz * iv;
  S.nlen = sqrtf(nb.x * nb.x + nb.y * nb.y + nb.z * nb.z);
  const float in = S.nlen > 0.f ? 1.0f / S.nlen : 0.f;
  S.nh[0] = nb.x * in;
  S.nh[1] = nb.y * in;
  S.nh[2] = nb.z * in;
  float hx = S.vh[0] + l[0], hy = S.vh[1] + l[1], hz = S.vh[2] + l[2];
  S.hlen = sqrtf(hx * hx + hy * hy + hz * hz);
  const float ih = S.hlen > 0.f ? 1.0f / S.hlen : 0.f;
  S.h[0] = hx * ih;
  S.h[1] = hy * ih;
  S.h[2] = hz * ih;
  S.nl = S.nh[0] * l[0] + S.nh[1] * l[1] + S.nh[2] * l[2];
  S.ndh = S.nh[0] * S.h[0] + S.nh[1] * S.h[1] + S.nh[2] * S.h[2];
  S.sd = k.x + k.y * fabsf(S.nl);
  S.ss = fabsf(S.nl) > 0.f ? k.z * powf(fabsf(S.ndh), nb.w) : 0.f;
  return S;
}

__global__ void __launch_bounds__(256)
    shade_kernel(LightSet ls, const float4* __restrict__ mean_v, const float4* __restrict__ nb,
                 const float4* __restrict__ kad, int64_t n, float2* __restrict__ out) {
  pdl_enter();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int v = blockIdx.y;
  const float4 m = mean_v[i];
  const ShadeTerms S = shade_terms(ls.l[v], ls.eye[v], make_float3(m.x, m.y, m.z), nb[i], kad[i]);
  out[(int64_t)v * n + i] = make_float2(S.sd, S.ss);
}

__global__ void __launch_bounds__(128)
    shade_bwd_kernel(LightSet ls, int n_views, const float4* __restrict__ mean_v,
                     const float4* __restrict__ nbv, const float4* __restrict__ kadv, int64_t n,
                     const int32_t* __restrict__ tiles, const float2* __restrict__ gshade,
                     float4* __restrict__ gmean, float4* __restrict__ gnb,
                     float4* __restrict__ gk) {
  pdl_enter();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 m = mean_v[i], nb = nbv[i], k = kadv[i];
  float dm[3] = {0.f, 0.f, 0.f}, dn[3] = {0.f, 0.f, 0.f};
  float dka = 0.f, dkd = 0.f, dks = 0.f, dbeta = 0.f;
  bool any = false;
  for (int v = 0; v < n_views; ++v) {
    const int64_t o = (int64_t)v * n + i;
    if (tiles[o] == 0) continue;
    const float2 g = gshade[o];
    if (g.x == 0.f && g.y == 0.f) continue;
    any = true;
    const float* l = ls.l[v];
    const ShadeTerms S = shade_terms(l, ls.eye[v], make_float3(m.x, m.y, m.z), nb, k);
    const float a = fabsf(S.ndh);
    const bool lit = fabsf(S.nl) > 0.f && a > 0.f;
    const float pw = lit ? powf(a, nb.w) : 0.f;
    const float dpw_da = lit ? nb.w * powf(a, nb.w - 1.0f) : 0.f;
    const float dpw_db = lit ? pw * logf(a) : 0.f;
    dka += g.x;
    dkd += g.x * fabsf(S.nl);
    dks += g.y * pw;
    dbeta += g.y * k.z * dpw_db;
    const float sgn_l = S.nl > 0.f ? 1.f : (S.nl < 0.f ? -1.f : 0.f);
    const float sgn_h = S.ndh > 0.f ? 1.f : (S.ndh < 0.f ? -1.f : 0.f);
    const float g_nl = g.x * k.y * sgn_l;
    const float g_ndh = g.y * k.z * dpw_da * sgn_h;
    float gn[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) gn[c] = g_nl * l[c] + g_ndh * S.h[c];
    const float pn = S.nh[0] * gn[0] + S.nh[1] * gn[1] + S.nh[2] * gn[2];
    const float in = S.nlen > 0.f ? 1.0f / S.nlen : 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) dn[c] += (gn[c] - S.nh[c] * pn) * in;
    // through h = (v_hat + l)/|v_hat + l| and v_hat = (eye - mu)/|eye - mu|
    float gh[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) gh[c] = g_ndh * S.nh[c];
    const float ph = S.h[0] * gh[0] + S.h[1] * gh[1] + S.h[2] * gh[2];
    const float ih = S.hlen > 0.f ? 1.0f / S.hlen : 0.f;
    float ghv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) ghv[c] = (gh[c] - S.h[c] * ph) * ih;
    const float pv = S.vh[0] * ghv[0] + S.vh[1] * ghv[1] + S.vh[2] * ghv[2];
    const float iv = S.vlen > 0.f ? 1.0f / S.vlen : 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) dm[c] -= (ghv[c] - S.vh[c] * pv) * iv;
  }
  if (!any) return;
  // add into the gradients with vector reductions (no read round trip)
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(gmean + i), "f"(dm[0]),
               "f"(dm[1]), "f"(dm[2]), "f"(0.0f) : "memory");
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(gnb + i), "f"(dn[0]),
               "f"(dn[1]), "f"(dn[2]), "f"(dbeta) : "memory");
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(gk + i), "f"(dka),
               "f"(dkd), "f"(dks), "f"(0.0f) : "memory");
}

veg_status fill_lights(const veg_camera* cams, int n_views, const float* light_dirs,
                       LightSet* out) {
  for (int v = 0; v < n_views; ++v) {
    const float* w = cams[v].world_to_cam;
    for (int c = 0; c < 3; ++c)  // eye = -R^T t
      out->eye[v][c] = -(w[0 * 4 + c] * w[3] + w[1 * 4 + c] * w[7] + w[2 * 4 + c] * w[11]);
    const float* l = light_dirs + 3 * v;
    const double len = std::sqrt((double)l[0] * l[0] + (double)l[1] * l[1] + (double)l[2] * l[2]);
    if (!(len > 0.0) || !std::isfinite(len)) return VEG_ERR_INVALID_ARGUMENT;
    for (int c = 0; c < 3; ++c) out->l[v][c] = (float)(l[c] / len);
  }
  return VEG_OK;
}

}  // namespace

}  // namespace veg

using namespace veg;

extern "C" veg_status veg_shade(const veg_camera* cams, int32_t n_views, const float* mean_v,
                                int64_t n, const float* normal_beta, const float* k_ads,
                                const float* light_dirs, float* splat_shade,
                                cudaStream_t stream) {
  veg_status st = check_cameras(cams, n_views);
  if (st != VEG_OK) return st;
  if (n < 0 || !light_dirs || n * n_views >= ((int64_t)1 << 31) ||
      (n > 0 && (!mean_v || !normal_beta || !k_ads || !splat_shade)))
    return VEG_ERR_INVALID_ARGUMENT;
  if (!aligned16(mean_v) || !aligned16(normal_beta) || !aligned16(k_ads) ||
      (reinterpret_cast<uintptr_t>(splat_shade) & 7))
    return VEG_ERR_INVALID_ARGUMENT;
  LightSet ls;
  st = fill_lights(cams, n_views, light_dirs, &ls);
  if (st != VEG_OK || n == 0) return st;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)n_views);
  launch_k(shade_kernel, grid, 256, 0, stream, 
      ls, reinterpret_cast<const float4*>(mean_v), reinterpret_cast<const float4*>(normal_beta),
      reinterpret_cast<const float4*>(k_ads), n, reinterpret_cast<float2*>(splat_shade));
  count_launch();
  return launch_status();
}

extern "C" veg_status veg_shade_bwd(const veg_camera* cams, int32_t n_views, const float* mean_v,
                                    int64_t n, const float* normal_beta, const float* k_ads,
                                    const float* light_dirs, const int32_t* tiles_touched,
                                    const float* grad_shade, float* grad_mean_v,
                                    float* grad_normal_beta, float* grad_k_ads,
                                    cudaStream_t stream) {
  veg_status st = check_cameras(cams, n_views);
  if (st != VEG_OK) return st;
  if (n < 0 || !light_dirs || n * n_views >= ((int64_t)1 << 31) ||
      (n > 0 && (!mean_v || !normal_beta || !k_ads || !tiles_touched || !grad_shade ||
                 !grad_mean_v || !grad_normal_beta || !grad_k_ads)))
    return VEG_ERR_INVALID_ARGUMENT;
  if (!aligned16(mean_v) || !aligned16(normal_beta) || !aligned16(k_ads) ||
      !aligned16(grad_mean_v) || !aligned16(grad_normal_beta) || !aligned16(grad_k_ads) ||
      (reinterpret_cast<uintptr_t>(grad_shade) & 7))
    return VEG_ERR_INVALID_ARGUMENT;
  LightSet ls;
  st = fill_lights(cams, n_views, light_dirs, &ls);
  if (st != VEG_OK || n == 0) return st;
  launch_k(shade_bwd_kernel, (unsigned)((n + 127) / 128), 128, 0, stream, 
      ls, n_views, reinterpret_cast<const float4*>(mean_v),
      reinterpret_cast<const float4*>(normal_beta), reinterpret_cast<const float4*>(k_ads), n,
      tiles_touched, reinterpret_cast<const float2*>(grad_shade),
      reinterpret_cast<float4*>(grad_mean_v), reinterpret_cast<float4*>(grad_normal_beta),
      reinterpret_cast<float4*>(grad_k_ads));
  count_launch();
  return launch_status();
}
