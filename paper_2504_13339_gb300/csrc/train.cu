// Training-side kernels (Sec. 4.2): the image loss (1 - lambda) L1 +
// lambda (1 - SSIM) with its gradient, and the Adam step on the Gaussians'
// raw parameters with the sigmoid activations of v and w.
//
// SSIM follows Wang et al. (2004): per colour channel, local means,
// variances and covariance under an 11 x 11 Gaussian window (sigma 1.5,
// normalised), zero padding at the image border, C1 = 0.01^2, C2 = 0.03^2.
// With S_q the index at pixel q and m1 = E[x], s11 = E[x^2], s12 = E[xy]
// its window statistics,
//   dS_q/dx_p = win(p - q) (dS_q/dm1 + 2 x_p dS_q/ds11 + y_p dS_q/ds12),
// so the gradient is three window sums of per-pixel partial derivatives.
//
// The statistics kernel computes S and the three partials once per pixel
// (16 x 16 tiles staging a 26 x 26 input region) and stores the partials in
// workspace planes; the gradient kernel filters the planes back.  Per-CTA
// sums of |x - y| and S go to the workspace and are reduced in a fixed order
// by a third kernel, so the loss is deterministic.
#include <cmath>

#include "veg_internal.cuh"

namespace veg {

namespace {

constexpr int kT = 16;             // output tile
constexpr int kR = 5;              // window radius
constexpr int kS = kT + 2 * kR;    // 26: a tile with the window's halo
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

struct Window {
  float w[2 * kR + 1];
};

// Two kernels per image, both on 16 x 16 tiles with a 5-pixel halo:
// l1_ssim_stats_kernel filters the five products (separable: rows, then
// columns; each thread four outputs from registers) for the tile's own
// pixels, forms S and its three partials there (per channel; written to
// workspace planes) and the per-tile sums of |x - y| and S;
// l1_ssim_grad_kernel filters the nine partial planes back (zero outside the
// image) and writes the combined gradient.  Every statistic is computed once
// per pixel instead of over an overlapping 26 x 26 region per tile.
constexpr int kB = 4;            // outputs per thread and pass
constexpr int kW = kB + 2 * kR;  // 14 values per thread and pass

struct StatsSmem {
  float x[3][kS * kS];  // inputs, per channel (zero outside the image)
  float y[3][kS * kS];
  float h[3][5][kS * kT];  // row pass of x, y, xx, yy, xy (26 rows x 16 columns)
};

struct GradSmem {
  float d[9][kS * kS];  // dS/dm1, dS/ds11, dS/ds12 per channel (zero outside the image)
  float e[9][kS * kT];  // row pass of the partials
  float g[9][kT * kT];  // column pass: the three window sums per channel
};

__global__ void __launch_bounds__(256)
    l1_ssim_stats_kernel(Window win, const float4* __restrict__ out, const float4* __restrict__ tgt,
                         int H, int W, int tiles_x, float* __restrict__ planes,
                         double2* __restrict__ partial) {
  pdl_enter();
  extern __shared__ float4 smem_raw[];
  StatsSmem& sm = *reinterpret_cast<StatsSmem*>(smem_raw);
  const int tid = threadIdx.x;
  const int tile = blockIdx.x, img = blockIdx.y;
  const int tx0 = (tile % tiles_x) * kT, ty0 = (tile / tiles_x) * kT;
  const int64_t HW = (int64_t)H * W, base = (int64_t)img * HW;
  for (int e = tid; e < kS * kS; e += 256) {
    const int r = e / kS, c = e - r * kS;
    const int gy = ty0 - kR + r, gx = tx0 - kR + c;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
      a = out[base + (int64_t)gy * W + gx];
      b = tgt[base + (int64_t)gy * W + gx];
    }
    sm.x[0][e] = a.x;
    sm.x[1][e] = a.y;
    sm.x[2][e] = a.z;
    sm.y[0][e] = b.x;
    sm.y[1][e] = b.y;
    sm.y[2][e] = b.z;
  }
  __syncthreads();
  // row pass of the five products: 3 channels x 26 rows x 4 segments
  for (int item = tid; item < 3 * kS * 4; item += 256) {
    const int ch = item / (kS * 4), rem = item - ch * (kS * 4);
    const int r = rem / 4, c0 = (rem % 4) * kB;
    const float* X = sm.x[ch];
    const float* Y = sm.y[ch];
    float xv[kW], yv[kW];
#pragma unroll
    for (int i = 0; i < kW; ++i) {
      xv[i] = X[r * kS + c0 + i];
      yv[i] = Y[r * kS + c0 + i];
    }
#pragma unroll
    for (int o = 0; o < kB; ++o) {
      float hx = 0.f, hy = 0.f, hxx = 0.f, hyy = 0.f, hxy = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * kR; ++k) {
        const float a = xv[o + k], b = yv[o + k], wk = win.w[k];
        hx = fmaf(wk, a, hx);
        hy = fmaf(wk, b, hy);
        hxx = fmaf(wk, a * a, hxx);
        hyy = fmaf(wk, b * b, hyy);
        hxy = fmaf(wk, a * b, hxy);
      }
      const int e = r * kT + c0 + o;
      sm.h[ch][0][e] = hx;
      sm.h[ch][1][e] = hy;
      sm.h[ch][2][e] = hxx;
      sm.h[ch][3][e] = hyy;
      sm.h[ch][4][e] = hxy;
    }
  }
  __syncthreads();
  // column pass: statistics, S and its partials at the tile's pixels,
  // 3 channels x 16 columns x 4 segments of four rows
  float ssum = 0.f;
  if (tid < 3 * kT * 4) {
    const int ch = tid / (kT * 4), rem = tid - ch * (kT * 4);
    const int c = rem % kT, r0 = (rem / kT) * kB;
    float st[5][kB];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      float hv[kW];
#pragma unroll
      for (int i = 0; i < kW; ++i) hv[i] = sm.h[ch][q][(r0 + i) * kT + c];
#pragma unroll
      for (int o = 0; o < kB; ++o) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * kR; ++k) acc = fmaf(win.w[k], hv[o + k], acc);
        st[q][o] = acc;
      }
    }
    const int gx = tx0 + c;
#pragma unroll
    for (int o = 0; o < kB; ++o) {
      const int gy = ty0 + r0 + o;
      if (gy >= H || gx >= W) continue;
      const float m1 = st[0][o], m2 = st[1][o], s11 = st[2][o], s22 = st[3][o];
      const float s12 = st[4][o];
      const float a1 = 2.f * m1 * m2 + kC1;
      const float a2 = 2.f * (s12 - m1 * m2) + kC2;
      const float b1 = m1 * m1 + m2 * m2 + kC1;
      const float b2 = (s11 - m1 * m1) + (s22 - m2 * m2) + kC2;
      const float ib = 1.0f / (b1 * b2);
      const float S = a1 * a2 * ib;
      const int64_t px = (int64_t)gy * W + gx;
      float* P = planes + ((int64_t)img * 9 + ch * 3) * HW + px;
      P[0] = 2.f * m2 * (a2 - a1) * ib - 2.f * m1 * S * (1.0f / b1 - 1.0f / b2);
      P[HW] = -S / b2;
      P[2 * HW] = 2.f * a1 * ib;
      ssum += S;
    }
  }
  // this thread's pixel: |x - y| over RGB
  float l1 = 0.f;
  {
    const int py = tid / kT, px = tid - py * kT;
    if (ty0 + py < H && tx0 + px < W) {
      const int io = (py + kR) * kS + px + kR;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) l1 += fabsf(sm.x[ch][io] - sm.y[ch][io]);
    }
  }
  // block sums of |x - y| and S (warp shuffles, then one thread)
  __shared__ float s_red[2][8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
    ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
  }
  if ((tid & 31) == 0) {
    s_red[0][tid >> 5] = l1;
    s_red[1][tid >> 5] = ssum;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < 8; ++w) {
      a += s_red[0][w];
      b += s_red[1][w];
    }
    partial[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = make_double2(a, b);
  }
}

__global__ void __launch_bounds__(256)
    l1_ssim_grad_kernel(Window win, const float4* __restrict__ out, const float4* __restrict__ tgt,
                        int H, int W, int tiles_x, float lam, float inv_count,
                        const float* __restrict__ planes, float4* __restrict__ grad) {
  pdl_enter();
  extern __shared__ float4 smem_raw[];
  GradSmem& sm = *reinterpret_cast<GradSmem*>(smem_raw);
  const int tid = threadIdx.x;
  const int tile = blockIdx.x, img = blockIdx.y;
  const int tx0 = (tile % tiles_x) * kT, ty0 = (tile / tiles_x) * kT;
  const int64_t HW = (int64_t)H * W, base = (int64_t)img * HW;
  for (int e = tid; e < 9 * kS * kS; e += 256) {
    const int q = e / (kS * kS), rem = e - q * (kS * kS);
    const int r = rem / kS, c = rem - r * kS;
    const int gy = ty0 - kR + r, gx = tx0 - kR + c;
    sm.d[q][rem] = (gy >= 0 && gy < H && gx >= 0 && gx < W)
                       ? planes[((int64_t)img * 9 + q) * HW + (int64_t)gy * W + gx]
                       : 0.f;
  }
  __syncthreads();
  // row pass of the partials: 9 planes x 26 rows x 4 segments
  for (int item = tid; item < 9 * kS * 4; item += 256) {
    const int q = item / (kS * 4), rem = item - q * (kS * 4);
    const int r = rem / 4, c0 = (rem % 4) * kB;
    float dv[kW];
#pragma unroll
    for (int i = 0; i < kW; ++i) dv[i] = sm.d[q][r * kS + c0 + i];
#pragma unroll
    for (int o = 0; o < kB; ++o) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * kR; ++k) acc = fmaf(win.w[k], dv[o + k], acc);
      sm.e[q][r * kT + c0 + o] = acc;
    }
  }
  __syncthreads();
  // column pass: 9 planes x 16 columns x 4 segments of four rows
  for (int item = tid; item < 9 * kT * 4; item += 256) {
    const int q = item / (kT * 4), rem = item - q * (kT * 4);
    const int c = rem % kT, r0 = (rem / kT) * kB;
    float ev[kW];
#pragma unroll
    for (int i = 0; i < kW; ++i) ev[i] = sm.e[q][(r0 + i) * kT + c];
#pragma unroll
    for (int o = 0; o < kB; ++o) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * kR; ++k) acc = fmaf(win.w[k], ev[o + k], acc);
      sm.g[q][(r0 + o) * kT + c] = acc;
    }
  }
  __syncthreads();
  // combine with the L1 part and write this thread's pixel
  const int py = tid / kT, px = tid - py * kT;
  if (ty0 + py < H && tx0 + px < W) {
    const int64_t o = base + (int64_t)(ty0 + py) * W + tx0 + px;
    const float4 a = out[o], b = tgt[o];
    const float xs[3] = {a.x, a.y, a.z}, ys[3] = {b.x, b.y, b.z};
    float gg[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const float g = sm.g[ch * 3][tid] + 2.f * xs[ch] * sm.g[ch * 3 + 1][tid] +
                      ys[ch] * sm.g[ch * 3 + 2][tid];
      const float diff = xs[ch] - ys[ch];
      const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
      gg[ch] = ((1.0f - lam) * sgn - lam * g) * inv_count;
    }
    grad[o] = make_float4(gg[0], gg[1], gg[2], 0.f);
  }
}

// Sums the per-CTA partials in a fixed order: loss[0] = (1 - lam) L1 +
// lam (1 - SSIM), loss[1] = L1, loss[2] = SSIM.
__global__ void __launch_bounds__(1024)
    l1_ssim_final_kernel(const double2* __restrict__ partial, int64_t n, double inv_count,
                         float lam, float* __restrict__ loss) {
  pdl_enter();
  __shared__ double s_a[1024], s_b[1024];
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    a += partial[i].x;
    b += partial[i].y;
  }
  s_a[threadIdx.x] = a;
  s_b[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s_a[threadIdx.x] += s_a[threadIdx.x + o];
      s_b[threadIdx.x] += s_b[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double l1 = s_a[0] * inv_count, ss = s_b[0] * inv_count;
    loss[0] = (float)((1.0 - lam) * l1 + lam * (1.0 - ss));
    loss[1] = (float)l1;
    loss[2] = (float)ss;
  }
}

// ---------------------------------------------------------------------------
// Adam (Kingma and Ba) on the raw parameters
// ---------------------------------------------------------------------------

struct AdamArgs {
  float4* param[5];
  const float4* grad[5];
  float4* m[5];
  float4* v[5];
  float4* rendered[2];
  float lr[5][4];
  float b1, b2, eps, inv_bc1, inv_sqrt_bc2;
  const veg_adam_counter* counter;  // bias corrections from here when set
};

__device__ __forceinline__ float sigmoid_f(float x) { return 1.0f / (1.0f + expf(-x)); }

__device__ __forceinline__ void adam_one(float& p, float& m, float& v, float g, float lr,
                                         const AdamArgs& A, float inv_bc1, float inv_sqrt_bc2) {
  m = A.b1 * m + (1.0f - A.b1) * g;
  v = A.b2 * v + (1.0f - A.b2) * g * g;
  p -= lr * (m * inv_bc1) / (sqrtf(v) * inv_sqrt_bc2 + A.eps);
}

// Advances the step counter and stores the step's bias corrections
// 1 / (1 - beta1^t) and 1 / sqrt(1 - beta2^t) (double, like the host path).
__global__ void adam_count_kernel(veg_adam_counter* c, float b1, float b2) {
  pdl_enter();
  const int64_t t = c->step + 1;
  c->step = t;
  c->inv_bc1 = (float)(1.0 / (1.0 - pow((double)b1, (double)t)));
  c->inv_sqrt_bc2 = (float)(1.0 / sqrt(1.0 - pow((double)b2, (double)t)));
}

__global__ void __launch_bounds__(256) adam_kernel(AdamArgs A, int64_t n) {
  pdl_enter();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  if (i >= n || A.param[a] == nullptr) return;
  const float inv_bc1 = A.counter ? A.counter->inv_bc1 : A.inv_bc1;
  const float inv_sqrt_bc2 = A.counter ? A.counter->inv_sqrt_bc2 : A.inv_sqrt_bc2;
  float4 p = A.param[a][i], g = A.grad[a][i], m = A.m[a][i], v = A.v[a][i];
  if (a < 2) {  // the fourth component is sigmoid-activated
    const float s = sigmoid_f(p.w);
    g.w *= s * (1.0f - s);
  }
  adam_one(p.x, m.x, v.x, g.x, A.lr[a][0], A, inv_bc1, inv_sqrt_bc2);
  adam_one(p.y, m.y, v.y, g.y, A.lr[a][1], A, inv_bc1, inv_sqrt_bc2);
  adam_one(p.z, m.z, v.z, g.z, A.lr[a][2], A, inv_bc1, inv_sqrt_bc2);
  adam_one(p.w, m.w, v.w, g.w, A.lr[a][3], A, inv_bc1, inv_sqrt_bc2);
  A.param[a][i] = p;
  A.m[a][i] = m;
  A.v[a][i] = v;
  if (a < 2 && A.rendered[a]) A.rendered[a][i] = make_float4(p.x, p.y, p.z, sigmoid_f(p.w));
}

// Workspace: per-tile (|x - y|, S) sums, then nine float planes per image
// (dS/dm1, dS/ds11, dS/ds12 per channel).
size_t loss_part_bytes(int64_t n_images, int H, int W) {
  return round_up((size_t)n_images * tiles_x_of(W) * tiles_x_of(H) * sizeof(double2), 256);
}
size_t loss_ws_bytes(int64_t n_images, int H, int W) {
  return loss_part_bytes(n_images, H, W) + (size_t)n_images * 9 * H * W * sizeof(float);
}

}  // namespace

}  // namespace veg

using namespace veg;

extern "C" veg_status veg_l1_ssim_loss_workspace_size(int64_t n_images, int32_t height,
                                                      int32_t width, size_t* bytes) {
  if (!bytes || n_images < 0 || height < 1 || width < 1 || height > 16384 || width > 16384)
    return VEG_ERR_INVALID_ARGUMENT;
  *bytes = loss_ws_bytes(n_images, height, width);
  return VEG_OK;
}

extern "C" veg_status veg_l1_ssim_loss(const float* out, const float* target, int64_t n_images,
                                       int32_t height, int32_t width, float lambda, float* grad,
                                       float* loss, void* workspace, size_t workspace_bytes,
                                       cudaStream_t stream) {
  if (n_images < 1 || height < 1 || width < 1 || height > 16384 || width > 16384 || !out ||
      !target || !grad || !loss || !workspace || !(lambda >= 0.f && lambda <= 1.f))
    return VEG_ERR_INVALID_ARGUMENT;
  if (!aligned16(out) || !aligned16(target) || !aligned16(grad) ||
      (reinterpret_cast<uintptr_t>(loss) & 3) || (reinterpret_cast<uintptr_t>(workspace) & 15))
    return VEG_ERR_INVALID_ARGUMENT;
  const int tx = tiles_x_of(width), ty = tiles_x_of(height);
  if (n_images > 65535 || workspace_bytes < loss_ws_bytes(n_images, height, width))
    return VEG_ERR_INVALID_ARGUMENT;
  Window win;
  double wsum = 0.0, wd[2 * kR + 1];
  for (int k = -kR; k <= kR; ++k)
    wsum += (wd[k + kR] = std::exp(-(double)k * k / (2.0 * 1.5 * 1.5)));
  for (int k = 0; k <= 2 * kR; ++k) win.w[k] = (float)(wd[k] / wsum);
  const double count = (double)n_images * height * width * 3.0;
  static SmemRecord cfg_stats, cfg_grad;
  veg_status st = prepare_smem(l1_ssim_stats_kernel, sizeof(StatsSmem), cfg_stats, false);
  if (st == VEG_OK) st = prepare_smem(l1_ssim_grad_kernel, sizeof(GradSmem), cfg_grad, false);
  if (st != VEG_OK) return st;
  double2* part = reinterpret_cast<double2*>(workspace);
  float* planes = reinterpret_cast<float*>(static_cast<char*>(workspace) +
                                           loss_part_bytes(n_images, height, width));
  const dim3 grid((unsigned)(tx * ty), (unsigned)n_images);
  const float4* o4 = reinterpret_cast<const float4*>(out);
  const float4* t4 = reinterpret_cast<const float4*>(target);
  launch_k(l1_ssim_stats_kernel, grid, 256, sizeof(StatsSmem), stream, win, o4, t4, height, width,
           tx, planes, part);
  launch_k(l1_ssim_grad_kernel, grid, 256, sizeof(GradSmem), stream, win, o4, t4, height, width,
           tx, lambda, (float)(1.0 / count), planes, reinterpret_cast<float4*>(grad));
  count_launch(2);
  launch_k(l1_ssim_final_kernel, 1, 1024, 0, stream, part, (int64_t)tx * ty * n_images, 1.0 / count,
                                               lambda, loss);
  count_launch();
  return launch_status();
}

namespace {

// The arrays and hyper-parameters of one step (step < 1: corrections from
// the device counter).
veg_status adam_args(const veg_adam_arrays* arrays, int64_t n, const float* lr, float beta1,
                     float beta2, float eps, int32_t step, AdamArgs& A) {
  if (!arrays || !lr || n < 0 || !(beta1 >= 0.f && beta1 < 1.f) ||
      !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f))
    return VEG_ERR_INVALID_ARGUMENT;
  for (int a = 0; a < 5; ++a) {
    A.param[a] = reinterpret_cast<float4*>(arrays->param[a]);
    A.grad[a] = reinterpret_cast<const float4*>(arrays->grad[a]);
    A.m[a] = reinterpret_cast<float4*>(arrays->exp_avg[a]);
    A.v[a] = reinterpret_cast<float4*>(arrays->exp_avg_sq[a]);
    if (A.param[a] && n > 0 && (!A.grad[a] || !A.m[a] || !A.v[a])) return VEG_ERR_INVALID_ARGUMENT;
    if (!aligned16(A.param[a]) || !aligned16(A.grad[a]) || !aligned16(A.m[a]) ||
        !aligned16(A.v[a]))
      return VEG_ERR_INVALID_ARGUMENT;
    for (int c = 0; c < 4; ++c) A.lr[a][c] = lr[a * 4 + c];
  }
  for (int a = 0; a < 2; ++a) {
    A.rendered[a] = reinterpret_cast<float4*>(arrays->rendered[a]);
    if (!aligned16(A.rendered[a])) return VEG_ERR_INVALID_ARGUMENT;
  }
  A.b1 = beta1;
  A.b2 = beta2;
  A.eps = eps;
  A.inv_bc1 = A.inv_sqrt_bc2 = 1.0f;
  if (step >= 1) {
    A.inv_bc1 = (float)(1.0 / (1.0 - std::pow((double)beta1, (double)step)));
    A.inv_sqrt_bc2 = (float)(1.0 / std::sqrt(1.0 - std::pow((double)beta2, (double)step)));
  }
  A.counter = nullptr;
  return VEG_OK;
}

}  // namespace

extern "C" veg_status veg_adam_step(const veg_adam_arrays* arrays, int64_t n, const float* lr,
                                    float beta1, float beta2, float eps, int32_t step,
                                    cudaStream_t stream) {
  if (step < 1) return VEG_ERR_INVALID_ARGUMENT;
  AdamArgs A;
  veg_status st = adam_args(arrays, n, lr, beta1, beta2, eps, step, A);
  if (st != VEG_OK || n == 0) return st;
  launch_k(adam_kernel, dim3((unsigned)((n + 255) / 256), 5), 256, 0, stream, A, n);
  count_launch();
  return launch_status();
}

extern "C" veg_status veg_adam_step_counted(const veg_adam_arrays* arrays, int64_t n,
                                            const float* lr, float beta1, float beta2, float eps,
                                            veg_adam_counter* counter, cudaStream_t stream) {
  if (!counter || (reinterpret_cast<uintptr_t>(counter) & 15)) return VEG_ERR_INVALID_ARGUMENT;
  AdamArgs A;
  veg_status st = adam_args(arrays, n, lr, beta1, beta2, eps, 0, A);
  if (st != VEG_OK) return st;
  A.counter = counter;
  launch_k(adam_count_kernel, 1, 1, 0, stream, counter, beta1, beta2);
  count_launch();
  if (n > 0) {
    launch_k(adam_kernel, dim3((unsigned)((n + 255) / 256), 5), 256, 0, stream, A, n);
    count_launch();
  }
  return launch_status();
}
