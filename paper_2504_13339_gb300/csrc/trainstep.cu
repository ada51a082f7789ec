// Native executor of one opacity-guided training iteration (Sec. 4.2): the
// library's own entry points issued in order from host code, so a training
// loop costs one call per iteration instead of one per stage.  It adds no
// arithmetic of its own; every stage is the entry point it names.
#include <cstring>

#include "veg_internal.cuh"

extern "C" veg_status veg_train_step(const veg_train_args* a, int32_t view, int32_t map,
                                     int32_t adam_step, int32_t accumulate_stats,
                                     cudaStream_t stream) {
  if (!a || !a->cams || view < 0 || view >= a->n_cams || map < 0 || map >= a->n_maps ||
      !a->luts || !a->targets || a->n < 0 || (a->lit && !a->light_dirs))
    return VEG_ERR_INVALID_ARGUMENT;
  const veg_camera* cam = a->cams + view;
  const int W = cam->width, H = cam->height;
  const int64_t img = (int64_t)W * H * 4;
  veg_tf tf;
  tf.lut = a->luts + (int64_t)map * a->lut_size * 4;
  tf.lut_size = a->lut_size;
  tf.n_tf = 1;
  tf.view_tf = nullptr;
  veg_gaussians g;
  g.mean_v = a->mean_v;
  g.logscale_w = a->logscale_w;
  g.quat = a->raw[2];
  g.n = a->n;
  veg_status st;
#define VEG_TRY(call)       \
  do {                      \
    st = (call);            \
    if (st != VEG_OK) return st; \
  } while (0)
  VEG_TRY(veg_project(cam, 1, g, &tf, a->splat_geo, a->splat_aux, a->tiles_touched, a->rect,
                      stream));
  const float* shade = nullptr;
  if (a->lit) {
    VEG_TRY(veg_shade(cam, 1, a->mean_v, a->n, a->raw[3], a->raw[4], a->light_dirs + 3 * view,
                      a->splat_shade, stream));
    shade = a->splat_shade;
  }
  VEG_TRY(veg_bin_sort(cam, 1, a->n, a->splat_geo, a->tiles_touched, a->rect, a->binsort_ws,
                       a->binsort_ws_bytes, a->capacity, nullptr, a->vals, a->tile_ranges,
                       stream));
  const int tiles = veg::tiles_x_of(W) * veg::tiles_x_of(H);
  VEG_TRY(veg_tile_order(a->tile_ranges, tiles, a->tile_order, stream));
  VEG_TRY(veg_composite_fwd(cam, 1, a->n, a->splat_geo, a->splat_aux, shade, a->vals,
                            a->tile_ranges, a->tile_order, tf, a->bg, a->tf_group, 0, a->out,
                            a->n_contrib, nullptr, stream));
  const float* target = a->targets + ((int64_t)view * a->n_maps + map) * img;
  VEG_TRY(veg_l1_ssim_loss(a->out, target, 1, H, W, a->lambda, a->loss_grad, a->loss,
                           a->loss_ws, a->loss_ws_bytes, stream));
  for (int k = 0; k < 5; ++k)
    if (a->grad[k] && a->n > 0 &&
        cudaMemsetAsync(a->grad[k], 0, (size_t)a->n * 16, stream) != cudaSuccess)
      return VEG_ERR_CUDA;
  VEG_TRY(veg_composite_bwd(cam, 1, g, a->splat_geo, a->splat_aux, shade, a->tiles_touched,
                            a->vals, a->tile_ranges, a->tile_order, tf, a->bg, a->tf_group, 0,
                            a->out, a->n_contrib, a->loss_grad, nullptr, 0, a->grad[0],
                            a->grad[1], a->grad[2], a->grad2d, a->lit ? a->grad_shade : nullptr,
                            nullptr, stream));
  if (a->lit)
    VEG_TRY(veg_shade_bwd(cam, 1, a->mean_v, a->n, a->raw[3], a->raw[4],
                          a->light_dirs + 3 * view, a->tiles_touched, a->grad_shade, a->grad[0],
                          a->grad[3], a->grad[4], stream));
  if (accumulate_stats && a->stat_accum)
    VEG_TRY(veg_grad_stats_accumulate(a->grad2d, a->tiles_touched, a->n, 1, W, H, a->stat_accum,
                                      a->stat_count, stream));
  if (adam_step >= 1) {
    veg_adam_arrays arr;
    std::memset(&arr, 0, sizeof(arr));
    for (int k = 0; k < 5; ++k) {
      arr.param[k] = a->raw[k];
      arr.grad[k] = a->grad[k];
      arr.exp_avg[k] = a->exp_avg[k];
      arr.exp_avg_sq[k] = a->exp_avg_sq[k];
    }
    arr.rendered[0] = a->mean_v;
    arr.rendered[1] = a->logscale_w;
    VEG_TRY(veg_adam_step(&arr, a->n, a->lr, a->beta1, a->beta2, a->eps, adam_step, stream));
  }
#undef VEG_TRY
  return VEG_OK;
}
