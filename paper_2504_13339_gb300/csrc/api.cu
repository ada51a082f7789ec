// Host-side glue of the C ABI: status strings, argument checks, the L1 loss
// kernels and the render convenience entry point.
#include <atomic>
#include <cmath>

#include "veg_internal.cuh"

namespace veg {

static std::atomic<uint64_t> g_launches{0};

void count_launch(int k) { g_launches.fetch_add((uint64_t)k, std::memory_order_relaxed); }

veg_status launch_status() {
  return cudaPeekAtLastError() == cudaSuccess ? VEG_OK : VEG_ERR_CUDA;
}

veg_status check_cameras(const veg_camera* cams, int32_t n_views) {
  if (!cams || n_views < 1 || n_views > VEG_MAX_VIEWS) return VEG_ERR_INVALID_ARGUMENT;
  for (int v = 0; v < n_views; ++v) {
    const veg_camera& c = cams[v];
    if (c.width < 1 || c.height < 1 || c.width > VEG_MAX_IMAGE || c.height > VEG_MAX_IMAGE)
      return VEG_ERR_INVALID_ARGUMENT;
    if (!(c.fx > 0.f) || !(c.fy > 0.f) || !std::isfinite(c.cx) || !std::isfinite(c.cy) ||
        !std::isfinite(c.near_plane))
      return VEG_ERR_INVALID_ARGUMENT;
    for (int k = 0; k < 12; ++k)
      if (!std::isfinite(c.world_to_cam[k])) return VEG_ERR_INVALID_ARGUMENT;
  }
  return VEG_OK;
}

veg_status check_cameras_one_size(const veg_camera* cams, int32_t n_views) {
  veg_status st = check_cameras(cams, n_views);
  if (st != VEG_OK) return st;
  for (int v = 1; v < n_views; ++v)
    if (cams[v].width != cams[0].width || cams[v].height != cams[0].height)
      return VEG_ERR_INVALID_ARGUMENT;
  return VEG_OK;
}

void fill_camset(const veg_camera* cams, int32_t n_views, CamSet* out) {
  for (int v = 0; v < n_views; ++v) {
    const veg_camera& c = cams[v];
    CamParam& p = out->c[v];
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) p.r[i * 3 + j] = c.world_to_cam[i * 4 + j];
      p.t[i] = c.world_to_cam[i * 4 + 3];
    }
    p.fx = c.fx;
    p.fy = c.fy;
    p.cx = c.cx;
    p.cy = c.cy;
    p.near_plane = c.near_plane;
    p.width = c.width;
    p.height = c.height;
    p.tiles_x = tiles_x_of(c.width);
    p.tiles_y = tiles_x_of(c.height);
  }
}

namespace {

constexpr int kLossBlocks = 1024;

__global__ void __launch_bounds__(256)
    l1_kernel(const float4* __restrict__ out, const float4* __restrict__ target, int64_t n,
              float inv_count, float4* __restrict__ grad, float* __restrict__ partials) {
  pdl_enter();
  __shared__ float s[256];
  float acc = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 o = out[i], t = target[i];
    const float dx = o.x - t.x, dy = o.y - t.y, dz = o.z - t.z;
    acc += fabsf(dx) + fabsf(dy) + fabsf(dz);
    grad[i] = make_float4((float)((dx > 0.f) - (dx < 0.f)) * inv_count,
                          (float)((dy > 0.f) - (dy < 0.f)) * inv_count,
                          (float)((dz > 0.f) - (dz < 0.f)) * inv_count, 0.f);
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(kLossBlocks)
    l1_final_kernel(const float* __restrict__ partials, float inv_count, float* __restrict__ loss) {
  pdl_enter();
  __shared__ double s[kLossBlocks];
  s[threadIdx.x] = (double)partials[threadIdx.x];
  __syncthreads();
  for (int o = kLossBlocks / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = (float)(s[0] * (double)inv_count);
}

struct RenderLayout {
  void* binsort_ws;
  size_t binsort_bytes;
  float4 *geo, *aux;
  int32_t* tiles;
  short4* rect;
  uint32_t* vals;
  int2* ranges;
  int32_t* order;
  size_t bytes;
};

RenderLayout carve_render(void* ws, int64_t n, int n_views, int64_t capacity,
                          int64_t total_tiles) {
  RenderLayout R;
  R.binsort_bytes = binsort_ws_bytes(n, n_views, capacity);
  Carver c(ws);
  R.binsort_ws = c.take<char>(R.binsort_bytes);  // first: its header is at offset 0
  R.geo = c.take<float4>((size_t)n * n_views);
  R.aux = c.take<float4>((size_t)n * n_views);
  R.tiles = c.take<int32_t>((size_t)n * n_views);
  R.rect = c.take<short4>((size_t)n * n_views);
  R.vals = c.take<uint32_t>((size_t)capacity);
  R.ranges = c.take<int2>((size_t)total_tiles);
  R.order = c.take<int32_t>((size_t)total_tiles);
  R.bytes = c.bytes();
  return R;
}

}  // namespace

}  // namespace veg

using namespace veg;

extern "C" const char* veg_status_string(veg_status status) {
  switch (status) {
    case VEG_OK: return "ok";
    case VEG_ERR_INVALID_ARGUMENT: return "invalid argument";
    case VEG_ERR_CAPACITY: return "tile-instance capacity exceeded";
    case VEG_ERR_CUDA: return "CUDA error";
    case VEG_ERR_TIMEOUT: return "device wait timed out";
    case VEG_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

extern "C" uint64_t veg_kernel_launches(void) { return g_launches.load(); }

extern "C" veg_status veg_l1_loss_workspace_size(size_t* bytes) {
  if (!bytes) return VEG_ERR_INVALID_ARGUMENT;
  *bytes = kLossBlocks * sizeof(float);
  return VEG_OK;
}

extern "C" veg_status veg_l1_loss(const float* out, const float* target, int64_t n_records,
                                  float* grad, float* loss, void* workspace,
                                  size_t workspace_bytes, cudaStream_t stream) {
  if (n_records < 0 || !loss || !workspace || workspace_bytes < kLossBlocks * sizeof(float))
    return VEG_ERR_INVALID_ARGUMENT;
  if (n_records > 0 && (!out || !target || !grad)) return VEG_ERR_INVALID_ARGUMENT;
  if (!aligned16(out) || !aligned16(target) || !aligned16(grad) ||
      (reinterpret_cast<uintptr_t>(workspace) & 3))
    return VEG_ERR_INVALID_ARGUMENT;
  const float inv = n_records > 0 ? (float)(1.0 / (3.0 * (double)n_records)) : 0.f;
  float* partials = static_cast<float*>(workspace);
  launch_k(l1_kernel, kLossBlocks, 256, 0, stream, reinterpret_cast<const float4*>(out),
                                             reinterpret_cast<const float4*>(target), n_records,
                                             inv, reinterpret_cast<float4*>(grad), partials);
  launch_k(l1_final_kernel, 1, kLossBlocks, 0, stream, partials, inv, loss);
  count_launch(2);
  return launch_status();
}

extern "C" veg_status veg_render_workspace_size(int64_t n, int32_t n_views, int64_t capacity,
                                                int32_t width, int32_t height, size_t* bytes) {
  if (!bytes || n < 0 || n_views < 1 || n_views > VEG_MAX_VIEWS || capacity < 0 ||
      capacity >= ((int64_t)1 << 31) || width < 1 || height < 1 || width > VEG_MAX_IMAGE ||
      height > VEG_MAX_IMAGE)
    return VEG_ERR_INVALID_ARGUMENT;
  // an upper bound for n_views views of at most width x height pixels
  *bytes = carve_render(nullptr, n, n_views, capacity,
                        (int64_t)n_views * tiles_x_of(width) * tiles_x_of(height))
               .bytes;
  return VEG_OK;
}

extern "C" veg_status veg_render(const veg_camera* cams, int32_t n_views, veg_gaussians g,
                                 veg_tf tf, const float* bg, int32_t tf_group, int64_t capacity,
                                 void* workspace, size_t workspace_bytes, float* out,
                                 int32_t* n_contrib, cudaStream_t stream) {
  veg_status st = check_cameras(cams, n_views);
  if (st != VEG_OK) return st;
  if (g.n < 0 || capacity < 0 || capacity >= ((int64_t)1 << 31) || !workspace || !out ||
      !n_contrib || !tf.lut || tf.lut_size < 2 || tf.n_tf < 1 || tf_group < 0 || tf_group > 8)
    return VEG_ERR_INVALID_ARGUMENT;
  const int64_t tiles = total_tiles_of(cams, n_views);
  if (tiles >= ((int64_t)1 << 31)) return VEG_ERR_INVALID_ARGUMENT;
  if (g.n * n_views >= ((int64_t)1 << 31)) return VEG_ERR_INVALID_ARGUMENT;
  if (g.n > 0 && (!g.mean_v || !g.logscale_w || !g.quat)) return VEG_ERR_INVALID_ARGUMENT;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) || !aligned16(out) || !aligned16(tf.lut) ||
      !aligned16(g.mean_v) || !aligned16(g.logscale_w) || !aligned16(g.quat))
    return VEG_ERR_INVALID_ARGUMENT;
  RenderLayout R = carve_render(workspace, g.n, n_views, capacity, tiles);
  if (workspace_bytes < R.bytes) return VEG_ERR_INVALID_ARGUMENT;
  CamSet cs;
  fill_camset(cams, n_views, &cs);
  st = project_launch(cs, n_views, g, &tf, R.geo, R.aux, R.tiles, R.rect, stream);
  if (st != VEG_OK) return st;
  st = binsort_launch(cams, n_views, g.n, R.geo, R.tiles, R.rect, R.binsort_ws, capacity, nullptr,
                      R.vals, R.ranges, stream);
  if (st != VEG_OK) return st;
  st = tile_order_launch(R.ranges, (int)tiles, R.order, stream);
  if (st != VEG_OK) return st;
  return composite_fwd_launch(cams, n_views, g.n, R.geo, R.aux, R.vals, R.ranges, R.order, tf, bg,
                              nullptr, tf_group, 0, reinterpret_cast<float4*>(out), n_contrib,
                              nullptr, stream);
}
