// Adaptive density control (Sec. 4.2, following 3D Gaussian splatting):
// the averaged view-space positional gradient per Gaussian, then clone,
// split and prune as one stream compaction that keeps the input order.
//
// Statistic: for each view where the Gaussian touches a tile, |(dL/du_x W/2,
// dL/du_y H/2)| (screen gradient in normalised device units) is added to a
// float32 accumulator and a count incremented, with every operation rounded
// separately so that the decisions are reproducible.
//
// Decisions (float32, thresholds prepared by the caller):
//   prune if w_raw < logit(w_min); else if accum / count >= g_min:
//   split if max(log-scale) > ln(dense_fraction * extent), clone otherwise;
//   else keep.
// Outputs in input order: keep -> 1 (moments kept), clone -> 2 (the copy
// with zero moments), split -> 2 children mu + R diag(s) z_j with log-scale
// - ln(split factor) and zero moments, prune -> 0.
#include <cmath>

#include "veg_internal.cuh"

namespace veg {

namespace {

constexpr int kItems = 4;                // items per thread
constexpr int kBlockItems = 256 * kItems;  // items per block

enum : int32_t { kPrune = 0, kKeep = 1, kClone = 2, kSplit = 3 };

__global__ void __launch_bounds__(256)
    grad_stats_kernel(const float4* __restrict__ grad2d, const int32_t* __restrict__ tiles,
                      int64_t n, int n_views, float hx, float hy, float* __restrict__ accum,
                      int32_t* __restrict__ count) {
  pdl_enter();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float a = accum[i];
  int32_t c = count[i];
  for (int v = 0; v < n_views; ++v) {
    const int64_t r = (int64_t)v * n + i;
    if (tiles[r] <= 0) continue;
    const float4 g = grad2d[2 * r];
    const float gx = mul(g.x, hx), gy = mul(g.y, hy);
    a = add(a, sqrt_rn(add(mul(gx, gx), mul(gy, gy))));
    ++c;
  }
  accum[i] = a;
  count[i] = c;
}

struct DensityArgs {
  const float4* in_p[5];
  const float4* in_m[5];
  const float4* in_v[5];
  float4* out_p[5];
  float4* out_m[5];
  float4* out_v[5];
  float4* rendered[2];
  const float* accum;
  const int32_t* count;
  const float* z;  // [n][2][3]
  float g_min, log_size, raw_w_min, log_split;
};

__device__ __forceinline__ int32_t classify_one(const DensityArgs& A, int64_t i) {
  const float4 lw = A.in_p[1][i];
  if (lw.w < A.raw_w_min) return kPrune;
  const int32_t c = A.count[i];
  const float avg = c > 0 ? dv(A.accum[i], (float)c) : 0.0f;
  if (!(avg >= A.g_min)) return kKeep;
  const float big = fmaxf(fmaxf(lw.x, lw.y), lw.z);
  return big > A.log_size ? kSplit : kClone;
}

__device__ __forceinline__ int outputs_of(int32_t act) { return act == kPrune ? 0 : act == kKeep ? 1 : 2; }

// Block-wide exclusive scan of one int per thread (256 threads); returns the
// prefix and writes the block total to *total.
__device__ __forceinline__ int block_exclusive_scan(int x, int* s_warp, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int w = lane < 8 ? s_warp[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < 8) s_warp[lane] = wi - w;  // exclusive warp offsets
    if (lane == 7) s_warp[8] = wi;
  }
  __syncthreads();
  const int res = s_warp[warp] + inc - x;
  *total = s_warp[8];
  return res;
}

__global__ void __launch_bounds__(256)
    density_classify_kernel(DensityArgs A, int64_t n, int32_t* __restrict__ action,
                            int64_t* __restrict__ block_sums) {
  pdl_enter();
  __shared__ int s_warp[9];
  const int64_t base = (int64_t)blockIdx.x * kBlockItems + (int64_t)threadIdx.x * kItems;
  int cnt = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int64_t i = base + k;
    if (i < n) {
      const int32_t a = classify_one(A, i);
      action[i] = a;
      cnt += outputs_of(a);
    }
  }
  int total;
  block_exclusive_scan(cnt, s_warp, &total);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// Exclusive scan of the block sums in one block (sequential chunks of 1024);
// writes the grand total to *n_out.
__global__ void __launch_bounds__(1024)
    density_scan_kernel(int64_t* __restrict__ block_sums, int64_t nb, int64_t* __restrict__ n_out) {
  pdl_enter();
  __shared__ int64_t s[1024];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
    const int64_t b = b0 + threadIdx.x;
    const int64_t x = b < nb ? block_sums[b] : 0;
    s[threadIdx.x] = x;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int64_t y = (int)threadIdx.x >= o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += y;
      __syncthreads();
    }
    if (b < nb) block_sums[b] = carry + s[threadIdx.x] - x;
    __syncthreads();
    if (threadIdx.x == 1023) carry += s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_out = carry;
}

__device__ __forceinline__ float sigmoid_d(float x) { return 1.0f / (1.0f + expf(-x)); }

__device__ void write_out(const DensityArgs& A, int64_t i, int64_t o, int child, bool keep_state) {
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 p0 = A.in_p[0][i], p1 = A.in_p[1][i];
  if (child >= 0) {
    // mu + R(q) diag(s) z for the normalised quaternion q = (w, x, y, z)
    const float4 q = A.in_p[2][i];
    const float qn = rsqrtf(q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z);
    const float w = q.x * qn, x = q.y * qn, y = q.z * qn, z = q.w * qn;
    const float* zz = A.z + (i * 2 + child) * 3;
    const float a = expf(p1.x) * zz[0], b = expf(p1.y) * zz[1], c = expf(p1.z) * zz[2];
    p0.x += (1.f - 2.f * (y * y + z * z)) * a + 2.f * (x * y - w * z) * b + 2.f * (x * z + w * y) * c;
    p0.y += 2.f * (x * y + w * z) * a + (1.f - 2.f * (x * x + z * z)) * b + 2.f * (y * z - w * x) * c;
    p0.z += 2.f * (x * z - w * y) * a + 2.f * (y * z + w * x) * b + (1.f - 2.f * (x * x + y * y)) * c;
    p1.x = sub(p1.x, A.log_split);
    p1.y = sub(p1.y, A.log_split);
    p1.z = sub(p1.z, A.log_split);
  }
#pragma unroll
  for (int a = 0; a < 5; ++a) {
    if (!A.in_p[a]) continue;
    A.out_p[a][o] = a == 0 ? p0 : a == 1 ? p1 : A.in_p[a][i];
    A.out_m[a][o] = keep_state ? A.in_m[a][i] : zero;
    A.out_v[a][o] = keep_state ? A.in_v[a][i] : zero;
  }
  if (A.rendered[0]) A.rendered[0][o] = make_float4(p0.x, p0.y, p0.z, sigmoid_d(p0.w));
  if (A.rendered[1]) A.rendered[1][o] = make_float4(p1.x, p1.y, p1.z, sigmoid_d(p1.w));
}

__global__ void __launch_bounds__(256)
    density_scatter_kernel(DensityArgs A, int64_t n, const int32_t* __restrict__ action,
                           const int64_t* __restrict__ block_offsets) {
  pdl_enter();
  __shared__ int s_warp[9];
  const int64_t base = (int64_t)blockIdx.x * kBlockItems + (int64_t)threadIdx.x * kItems;
  int32_t act[kItems];
  int cnt = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int64_t i = base + k;
    act[k] = i < n ? action[i] : kPrune;
    cnt += outputs_of(act[k]);
  }
  int total;
  int64_t o = block_offsets[blockIdx.x] + block_exclusive_scan(cnt, s_warp, &total);
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int64_t i = base + k;
    if (act[k] == kKeep) {
      write_out(A, i, o, -1, true);
    } else if (act[k] == kClone) {
      write_out(A, i, o, -1, true);
      write_out(A, i, o + 1, -1, false);
    } else if (act[k] == kSplit) {
      write_out(A, i, o, 0, false);
      write_out(A, i, o + 1, 1, false);
    }
    o += outputs_of(act[k]);
  }
}

size_t density_ws_bytes(int64_t n) {
  Carver c(nullptr);
  c.take<int32_t>((size_t)n);
  c.take<int64_t>((size_t)((n + kBlockItems - 1) / kBlockItems) + 1);
  return c.bytes();
}

}  // namespace

}  // namespace veg

using namespace veg;

extern "C" veg_status veg_grad_stats_accumulate(const float* grad2d, const int32_t* tiles_touched,
                                                int64_t n, int32_t n_views, int32_t width,
                                                int32_t height, float* accum, int32_t* count,
                                                cudaStream_t stream) {
  if (n < 0 || n_views < 1 || n_views > VEG_MAX_VIEWS || width < 1 || height < 1 ||
      n * n_views >= ((int64_t)1 << 31))
    return VEG_ERR_INVALID_ARGUMENT;
  if (n > 0 && (!grad2d || !tiles_touched || !accum || !count)) return VEG_ERR_INVALID_ARGUMENT;
  if (!aligned16(grad2d) || (reinterpret_cast<uintptr_t>(accum) & 3) ||
      (reinterpret_cast<uintptr_t>(count) & 3))
    return VEG_ERR_INVALID_ARGUMENT;
  if (n == 0) return VEG_OK;
  launch_k(grad_stats_kernel, (unsigned)((n + 255) / 256), 256, 0, stream, 
      reinterpret_cast<const float4*>(grad2d), tiles_touched, n, n_views, 0.5f * (float)width,
      0.5f * (float)height, accum, count);
  count_launch();
  return launch_status();
}

extern "C" veg_status veg_densify_workspace_size(int64_t n, size_t* bytes) {
  if (!bytes || n < 0) return VEG_ERR_INVALID_ARGUMENT;
  *bytes = density_ws_bytes(n);
  return VEG_OK;
}

extern "C" veg_status veg_densify(const veg_adam_arrays* in, int64_t n, const float* accum,
                                  const int32_t* count, const float* split_normals,
                                  veg_density_config cfg, const veg_adam_arrays* out,
                                  int64_t out_capacity, int64_t* n_out, int32_t* action,
                                  void* workspace, size_t workspace_bytes, cudaStream_t stream) {
  if (!in || !out || !n_out || n < 0 || out_capacity < 2 * n) return VEG_ERR_INVALID_ARGUMENT;
  if (n > 0 && (!accum || !count || !split_normals || !in->param[0] || !in->param[1] ||
                !in->param[2]))
    return VEG_ERR_INVALID_ARGUMENT;
  if (!workspace || workspace_bytes < density_ws_bytes(n) ||
      (reinterpret_cast<uintptr_t>(workspace) & 255) || (reinterpret_cast<uintptr_t>(n_out) & 7))
    return VEG_ERR_INVALID_ARGUMENT;
  DensityArgs A;
  for (int a = 0; a < 5; ++a) {
    A.in_p[a] = reinterpret_cast<const float4*>(in->param[a]);
    A.in_m[a] = reinterpret_cast<const float4*>(in->exp_avg[a]);
    A.in_v[a] = reinterpret_cast<const float4*>(in->exp_avg_sq[a]);
    A.out_p[a] = reinterpret_cast<float4*>(out->param[a]);
    A.out_m[a] = reinterpret_cast<float4*>(out->exp_avg[a]);
    A.out_v[a] = reinterpret_cast<float4*>(out->exp_avg_sq[a]);
    if (A.in_p[a] && (!A.in_m[a] || !A.in_v[a] || !A.out_p[a] || !A.out_m[a] || !A.out_v[a]))
      return VEG_ERR_INVALID_ARGUMENT;
    if (!aligned16(A.in_p[a]) || !aligned16(A.in_m[a]) || !aligned16(A.in_v[a]) ||
        !aligned16(A.out_p[a]) || !aligned16(A.out_m[a]) || !aligned16(A.out_v[a]))
      return VEG_ERR_INVALID_ARGUMENT;
  }
  for (int a = 0; a < 2; ++a) {
    A.rendered[a] = reinterpret_cast<float4*>(out->rendered[a]);
    if (!aligned16(A.rendered[a])) return VEG_ERR_INVALID_ARGUMENT;
  }
  A.accum = accum;
  A.count = count;
  A.z = split_normals;
  A.g_min = cfg.grad_threshold;
  A.log_size = cfg.log_size_threshold;
  A.raw_w_min = cfg.raw_weight_threshold;
  A.log_split = cfg.log_split_factor;
  const int64_t nb = (n + kBlockItems - 1) / kBlockItems;
  Carver c(workspace);
  int32_t* act_ws = c.take<int32_t>((size_t)n);
  int64_t* sums = c.take<int64_t>((size_t)nb + 1);
  int32_t* act = action ? action : act_ws;
  if (n == 0) {
    if (cudaMemsetAsync(n_out, 0, sizeof(int64_t), stream) != cudaSuccess) return VEG_ERR_CUDA;
    return VEG_OK;
  }
  launch_k(density_classify_kernel, (unsigned)nb, 256, 0, stream, A, n, act, sums);
  launch_k(density_scan_kernel, 1, 1024, 0, stream, sums, nb, n_out);
  launch_k(density_scatter_kernel, (unsigned)nb, 256, 0, stream, A, n, act, sums);
  count_launch(3);
  return launch_status();
}
