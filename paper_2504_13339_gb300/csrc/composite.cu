// Entry points of the compositing stage: forward (Eq. 1) for a group of
// transfer functions per pass, and the backward pass through the blend, the
// transfer function and (optionally) the projection.
#include "composite_kernels.cuh"

namespace veg {

veg_status project_bwd_launch(const CamSet& cs, int n_views, veg_gaussians g,
                              const int32_t* tiles, const float4* grad2d, float4* gm, float4* gl,
                              float4* gq, cudaStream_t stream, int64_t first = 0,
                              int64_t count = -1);

veg_status composite_fwd_launch(const veg_camera* cams, int n_views, int64_t n,
                                const float4* geo, const float4* aux, const uint32_t* vals,
                                const int2* ranges, const int32_t* order, veg_tf tf,
                                const float* bg, const float* shade, int tf_group,
                                int tile_batch, float4* out, int32_t* n_contrib,
                                unsigned long long* stats, cudaStream_t stream) {
  CompArgs A = make_args(cams, n_views, geo, aux, vals, ranges, order, tf, bg, shade);
  (void)n;
  const int B = pick_batch(tile_batch);
  const int TG = tf.view_tf ? 1
                            : pick_group(tf_group, tf.n_tf, false, tf.lut_size, shade != nullptr,
                                         stats ? 256 : B);
  if (shade) {
    if (stats) return VEG_ERR_UNSUPPORTED;
    switch (TG) {
      case 1: return fwd_batch<1, false, true>(B, A, n_views, out, n_contrib, nullptr, stream);
      case 2: return fwd_batch<2, false, true>(B, A, n_views, out, n_contrib, nullptr, stream);
      case 4: return fwd_batch<4, false, true>(B, A, n_views, out, n_contrib, nullptr, stream);
      default: return fwd_batch<8, false, true>(B, A, n_views, out, n_contrib, nullptr, stream);
    }
  }
  if (stats) {
    switch (TG) {
      case 1: return fwd_batch<1, true, false>(B, A, n_views, out, n_contrib, stats, stream);
      case 2: return fwd_batch<2, true, false>(B, A, n_views, out, n_contrib, stats, stream);
      case 4: return fwd_batch<4, true, false>(B, A, n_views, out, n_contrib, stats, stream);
      default: return fwd_batch<8, true, false>(B, A, n_views, out, n_contrib, stats, stream);
    }
  }
  switch (TG) {
    case 1: return fwd_batch<1, false, false>(B, A, n_views, out, n_contrib, nullptr, stream);
    case 2: return fwd_batch<2, false, false>(B, A, n_views, out, n_contrib, nullptr, stream);
    case 4: return fwd_batch<4, false, false>(B, A, n_views, out, n_contrib, nullptr, stream);
    default: return fwd_batch<8, false, false>(B, A, n_views, out, n_contrib, nullptr, stream);
  }
}

size_t composite_bwd_ws_bytes(int64_t n, int n_views) {
  Carver c(nullptr);
  c.take<float4>((size_t)2 * n * n_views);
  return c.bytes();
}

}  // namespace veg

using namespace veg;

static bool batch_ok(int32_t b) { return b == 0 || b == 128 || b == 256 || b == 512; }

static veg_status check_composite_common(const veg_camera* cams, int32_t n_views, int64_t n,
                                         const float* geo, const float* aux, const uint32_t* vals,
                                         const int32_t* ranges, veg_tf tf) {
  veg_status st = check_cameras(cams, n_views);
  if (st != VEG_OK) return st;
  if (n < 0 || !ranges || !tf.lut || tf.lut_size < 2 || tf.n_tf < 1 || tf.n_tf > 4096)
    return VEG_ERR_INVALID_ARGUMENT;
  if (total_tiles_of(cams, n_views) >= ((int64_t)1 << 31)) return VEG_ERR_INVALID_ARGUMENT;
  if (tf.lut_size > 4096) return VEG_ERR_UNSUPPORTED;
  if (n > 0 && (!geo || !aux || !vals)) return VEG_ERR_INVALID_ARGUMENT;
  if (!aligned16(geo) || !aligned16(aux) || !aligned16(tf.lut) ||
      (reinterpret_cast<uintptr_t>(ranges) & 7))
    return VEG_ERR_INVALID_ARGUMENT;
  return VEG_OK;
}

extern "C" veg_status veg_composite_fwd(const veg_camera* cams, int32_t n_views, int64_t n,
                                        const float* splat_geo, const float* splat_aux,
                                        const float* splat_shade, const uint32_t* vals,
                                        const int32_t* tile_ranges, const int32_t* tile_order,
                                        veg_tf tf, const float* bg, int32_t tf_group,
                                        int32_t tile_batch, float* out, int32_t* n_contrib,
                                        unsigned long long* stats, cudaStream_t stream) {
  veg_status st =
      check_composite_common(cams, n_views, n, splat_geo, splat_aux, vals, tile_ranges, tf);
  if (st != VEG_OK) return st;
  if (!out || !n_contrib || !aligned16(out) || tf_group < 0 || tf_group > 8 ||
      !batch_ok(tile_batch) || (reinterpret_cast<uintptr_t>(splat_shade) & 7))
    return VEG_ERR_INVALID_ARGUMENT;
  return composite_fwd_launch(cams, n_views, n, reinterpret_cast<const float4*>(splat_geo),
                              reinterpret_cast<const float4*>(splat_aux), vals,
                              reinterpret_cast<const int2*>(tile_ranges), tile_order, tf, bg,
                              splat_shade, tf_group, tile_batch, reinterpret_cast<float4*>(out),
                              n_contrib, stats, stream);
}

extern "C" veg_status veg_composite_bwd_workspace_size(int64_t n, int32_t n_views,
                                                       size_t* bytes) {
  if (!bytes || n < 0 || n_views < 1 || n_views > VEG_MAX_VIEWS) return VEG_ERR_INVALID_ARGUMENT;
  *bytes = composite_bwd_ws_bytes(n, n_views);
  return VEG_OK;
}

extern "C" veg_status veg_composite_bwd(const veg_camera* cams, int32_t n_views, veg_gaussians g,
                                        const float* splat_geo, const float* splat_aux,
                                        const float* splat_shade,
                                        const int32_t* tiles_touched, const uint32_t* vals,
                                        const int32_t* tile_ranges, const int32_t* tile_order,
                                        veg_tf tf, const float* bg, int32_t tf_group,
                                        int32_t tile_batch, const float* out,
                                        const int32_t* n_contrib, const float* dL_dout,
                                        void* workspace, size_t workspace_bytes,
                                        float* grad_mean_v, float* grad_logscale_w,
                                        float* grad_quat, float* grad2d, float* grad_shade,
                                        unsigned long long* stats, cudaStream_t stream) {
  veg_status st =
      check_composite_common(cams, n_views, g.n, splat_geo, splat_aux, vals, tile_ranges, tf);
  if (st != VEG_OK) return st;
  if (!out || !n_contrib || !dL_dout || !aligned16(out) || !aligned16(dL_dout) || tf_group < 0 ||
      tf_group > 8 || !batch_ok(tile_batch))
    return VEG_ERR_INVALID_ARGUMENT;
  const bool only_2d = !grad_mean_v && !grad_logscale_w && !grad_quat;
  if (only_2d && !grad2d) return VEG_ERR_INVALID_ARGUMENT;
  if (g.n > 0 && !only_2d &&
      (!g.mean_v || !g.logscale_w || !g.quat || !tiles_touched || !grad_mean_v ||
       !grad_logscale_w || !grad_quat))
    return VEG_ERR_INVALID_ARGUMENT;
  if (!aligned16(grad_mean_v) || !aligned16(grad_logscale_w) || !aligned16(grad_quat) ||
      !aligned16(grad2d) || !aligned16(g.mean_v) || !aligned16(g.logscale_w) ||
      !aligned16(g.quat))
    return VEG_ERR_INVALID_ARGUMENT;
  const bool lit = splat_shade != nullptr;
  if (lit && (!grad_shade || (reinterpret_cast<uintptr_t>(splat_shade) & 7) ||
              (reinterpret_cast<uintptr_t>(grad_shade) & 7)))
    return VEG_ERR_INVALID_ARGUMENT;
  if (lit && stats) return VEG_ERR_UNSUPPORTED;
  float4* g2 = reinterpret_cast<float4*>(grad2d);
  if (!g2) {
    if (!workspace || workspace_bytes < composite_bwd_ws_bytes(g.n, n_views) ||
        (reinterpret_cast<uintptr_t>(workspace) & 255))
      return VEG_ERR_INVALID_ARGUMENT;
    g2 = reinterpret_cast<float4*>(workspace);
  }
  const int64_t nrec2 = 2 * g.n * n_views;
  if (nrec2 > 0 && cudaMemsetAsync(g2, 0, (size_t)nrec2 * sizeof(float4), stream) != cudaSuccess)
    return VEG_ERR_CUDA;
  float2* gsh = reinterpret_cast<float2*>(grad_shade);
  if (lit && nrec2 > 0 &&
      cudaMemsetAsync(gsh, 0, (size_t)(nrec2 / 2) * sizeof(float2), stream) != cudaSuccess)
    return VEG_ERR_CUDA;
  CompArgs A = make_args(cams, n_views, reinterpret_cast<const float4*>(splat_geo),
                         reinterpret_cast<const float4*>(splat_aux), vals,
                         reinterpret_cast<const int2*>(tile_ranges), tile_order, tf, bg,
                         splat_shade);
  const int B = pick_batch(tile_batch);
  const int TG = tf.view_tf ? 1
                            : pick_group(tf_group, tf.n_tf, true, tf.lut_size, lit,
                                         stats ? 256 : B);
  const float4* o4 = reinterpret_cast<const float4*>(out);
  const float4* d4 = reinterpret_cast<const float4*>(dL_dout);
  if (lit) {
    switch (TG) {
      case 1: st = bwd_batch<1, false, true>(B, A, n_views, o4, n_contrib, d4, g2, gsh, nullptr, stream); break;
      case 2: st = bwd_batch<2, false, true>(B, A, n_views, o4, n_contrib, d4, g2, gsh, nullptr, stream); break;
      default: st = bwd_batch<4, false, true>(B, A, n_views, o4, n_contrib, d4, g2, gsh, nullptr, stream); break;
    }
  } else if (stats) {
    switch (TG) {
      case 1: st = bwd_batch<1, true, false>(B, A, n_views, o4, n_contrib, d4, g2, nullptr, stats, stream); break;
      case 2: st = bwd_batch<2, true, false>(B, A, n_views, o4, n_contrib, d4, g2, nullptr, stats, stream); break;
      default: st = bwd_batch<4, true, false>(B, A, n_views, o4, n_contrib, d4, g2, nullptr, stats, stream); break;
    }
  } else {
    switch (TG) {
      case 1: st = bwd_batch<1, false, false>(B, A, n_views, o4, n_contrib, d4, g2, nullptr, nullptr, stream); break;
      case 2: st = bwd_batch<2, false, false>(B, A, n_views, o4, n_contrib, d4, g2, nullptr, nullptr, stream); break;
      default: st = bwd_batch<4, false, false>(B, A, n_views, o4, n_contrib, d4, g2, nullptr, nullptr, stream); break;
    }
  }
  if (st != VEG_OK || only_2d) return st;
  CamSet cs;
  fill_camset(cams, n_views, &cs);
  return project_bwd_launch(cs, n_views, g, tiles_touched, g2,
                            reinterpret_cast<float4*>(grad_mean_v),
                            reinterpret_cast<float4*>(grad_logscale_w),
                            reinterpret_cast<float4*>(grad_quat), stream);
}

namespace {
veg_status project_bwd_checked(const veg_camera* cams, int32_t n_views, veg_gaussians g,
                               const int32_t* tiles_touched, const float* grad2d, int64_t first,
                               int64_t count, float* grad_mean_v, float* grad_logscale_w,
                               float* grad_quat, cudaStream_t stream) {
  veg_status st = check_cameras(cams, n_views);
  if (st != VEG_OK) return st;
  if (g.n < 0 || g.n * n_views >= ((int64_t)1 << 31)) return VEG_ERR_INVALID_ARGUMENT;
  if (first < 0 || count < 0 || first > g.n || count > g.n - first)
    return VEG_ERR_INVALID_ARGUMENT;
  if (count > 0 && (!g.mean_v || !g.logscale_w || !g.quat || !tiles_touched || !grad2d ||
                    !grad_mean_v || !grad_logscale_w || !grad_quat))
    return VEG_ERR_INVALID_ARGUMENT;
  if (!aligned16(grad2d) || !aligned16(grad_mean_v) || !aligned16(grad_logscale_w) ||
      !aligned16(grad_quat) || !aligned16(g.mean_v) || !aligned16(g.logscale_w) ||
      !aligned16(g.quat))
    return VEG_ERR_INVALID_ARGUMENT;
  CamSet cs;
  fill_camset(cams, n_views, &cs);
  return project_bwd_launch(cs, n_views, g, tiles_touched,
                            reinterpret_cast<const float4*>(grad2d),
                            reinterpret_cast<float4*>(grad_mean_v),
                            reinterpret_cast<float4*>(grad_logscale_w),
                            reinterpret_cast<float4*>(grad_quat), stream, first, count);
}
}  // namespace

extern "C" veg_status veg_project_bwd(const veg_camera* cams, int32_t n_views, veg_gaussians g,
                                      const int32_t* tiles_touched, const float* grad2d,
                                      float* grad_mean_v, float* grad_logscale_w,
                                      float* grad_quat, cudaStream_t stream) {
  return project_bwd_checked(cams, n_views, g, tiles_touched, grad2d, 0, g.n < 0 ? 0 : g.n,
                             grad_mean_v, grad_logscale_w, grad_quat, stream);
}

extern "C" veg_status veg_project_bwd_range(const veg_camera* cams, int32_t n_views,
                                            veg_gaussians g, const int32_t* tiles_touched,
                                            const float* grad2d, int64_t first, int64_t count,
                                            float* grad_mean_v, float* grad_logscale_w,
                                            float* grad_quat, cudaStream_t stream) {
  return project_bwd_checked(cams, n_views, g, tiles_touched, grad2d, first, count, grad_mean_v,
                             grad_logscale_w, grad_quat, stream);
}
