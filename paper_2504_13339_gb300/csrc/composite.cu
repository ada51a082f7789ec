// Front-to-back compositing (Eq. 1) of depth-sorted splats per 16x16 tile,
// for several transfer functions per pass, and its backward pass.
//
// One CTA of 256 threads owns one (view, tile, TF group); each thread owns
// one pixel (warps cover 8x4 pixel blocks).  The tile's list is staged in
// batches of 256 splats through shared memory: the stager evaluates every
// splat's colour and opacity under each TF of the group once (linear
// interpolation in the TF tables, which sit in shared memory), so the
// per-pixel inner loop is one 2D Gaussian evaluation shared by the group
// plus a handful of FP32 operations per TF.  A pixel leaves the loop once
// every TF of the group has terminated (T (1 - alpha) < 1e-4); the block
// stops staging when all its pixels have left.
//
// The per-pair arithmetic that decides skips, the 0.99 clamp and
// termination is written with explicitly rounded operations and shared by
// the forward and backward kernels, so the backward replays the forward's
// decisions bit for bit.
#include <algorithm>

#include "veg_internal.cuh"

namespace veg {

namespace {

constexpr int kBatch = 256;

// 2^x with the hardware approximation (ex2.approx.ftz), x = power * log2(e).
__device__ __forceinline__ float gauss_of(float power) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(mul(power, 1.44269502162933349609375f)));
  return fminf(y, 1.0f);
}

// power = -1/2 (a dx^2 + c dy^2) - b dx dy with (na, nb, nc) = (-a/2, -b, -c/2).
__device__ __forceinline__ float power_of(float dx, float dy, float na, float nb, float nc) {
  return __fmaf_rn(na, mul(dx, dx), __fmaf_rn(nc, mul(dy, dy), mul(nb, mul(dx, dy))));
}

__device__ __forceinline__ void pixel_of(int tile, int tiles_x, int& px, int& py) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  px = (tile % tiles_x) * VEG_TILE + (w & 1) * 8 + (l & 7);
  py = (tile / tiles_x) * VEG_TILE + (w >> 1) * 4 + (l >> 3);
}

struct CompArgs {
  const float4* geo;
  const float4* aux;
  const uint32_t* vals;
  const int2* ranges;
  const float4* lut;
  int lut_size, n_tf;
  int width, height, tiles_x, tiles_per_view;
  float bg0, bg1, bg2;
};

// Loads the TF tables of group [t0, t0+TG) into shared memory (missing
// tables read as fully transparent).
template <int TG>
__device__ __forceinline__ void stage_luts(const CompArgs& A, int t0, float4* s_lut) {
  const int L = A.lut_size;
  for (int e = threadIdx.x; e < TG * L; e += blockDim.x) {
    int t = e / L, k = e - t * L;
    s_lut[e] = (t0 + t < A.n_tf) ? __ldg(&A.lut[(int64_t)(t0 + t) * L + k])
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

template <int TG, bool STATS>
__global__ void __launch_bounds__(256)
    composite_fwd_kernel(CompArgs A, float4* __restrict__ out, int32_t* __restrict__ n_contrib,
                         unsigned long long* __restrict__ stats) {
  extern __shared__ float4 s_lut[];  // [TG][L]
  __shared__ float4 s_geo[kBatch];   // u_x, u_y, -a/2, -b
  __shared__ float s_c[kBatch];      // -c/2
  __shared__ float4 s_col[TG][kBatch];
  const int tile = blockIdx.x, view = blockIdx.y, t0 = blockIdx.z * TG;
  const int ntg = min(TG, A.n_tf - t0);
  stage_luts<TG>(A, t0, s_lut);
  int px, py;
  pixel_of(tile, A.tiles_x, px, py);
  const bool inside = px < A.width && py < A.height;
  const float fx = (float)px, fy = (float)py;
  const int2 rg = A.ranges[(int64_t)view * A.tiles_per_view + tile];
  float T[TG], Cr[TG], Cg[TG], Cb[TG];
  int last[TG];
#pragma unroll
  for (int t = 0; t < TG; ++t) {
    T[t] = 1.0f;
    Cr[t] = Cg[t] = Cb[t] = 0.0f;
    last[t] = 0;
  }
  unsigned act = inside ? ((1u << ntg) - 1u) : 0u;
  unsigned long long n_vis = 0, n_alpha = 0, n_blend = 0;
  const int L = A.lut_size;

  for (int start = rg.x; start < rg.y; start += kBatch) {
    if (__syncthreads_count(act != 0u) == 0) break;
    const int i = start + threadIdx.x;
    if (i < rg.y) {
      const uint32_t g = A.vals[i];
      const float4 ge = A.geo[g], au = A.aux[g];
      s_geo[threadIdx.x] = make_float4(ge.x, ge.y, -0.5f * au.x, -au.y);
      s_c[threadIdx.x] = -0.5f * au.z;
      const TfPos q = tf_pos(au.w, L);
#pragma unroll
      for (int t = 0; t < TG; ++t) {
        const float4 lo = s_lut[t * L + q.k], hi = s_lut[t * L + q.k + 1];
        s_col[t][threadIdx.x] = make_float4(lerp_rn(lo.x, hi.x, q), lerp_rn(lo.y, hi.y, q),
                                            lerp_rn(lo.z, hi.z, q),
                                            mul(lerp_rn(lo.w, hi.w, q), ge.w));
      }
    }
    __syncthreads();
    const int cnt = min(kBatch, rg.y - start);
    for (int j = 0; j < cnt && act; ++j) {
      const float4 sg = s_geo[j];
      const float power = power_of(sub(sg.x, fx), sub(sg.y, fy), sg.z, sg.w, s_c[j]);
      if (STATS) ++n_vis;
      if (power > 0.0f) continue;
      const float G = gauss_of(power);
#pragma unroll
      for (int t = 0; t < TG; ++t) {
        if (!(act & (1u << t))) continue;
        if (STATS) ++n_alpha;
        const float4 c = s_col[t][j];
        const float alpha = fminf(kAlphaMax, mul(c.w, G));
        if (alpha < kAlphaMin) continue;
        const float test = mul(T[t], sub(1.0f, alpha));
        if (test < kTMin) {
          act &= ~(1u << t);
          continue;
        }
        const float wgt = mul(alpha, T[t]);
        Cr[t] = __fmaf_rn(c.x, wgt, Cr[t]);
        Cg[t] = __fmaf_rn(c.y, wgt, Cg[t]);
        Cb[t] = __fmaf_rn(c.z, wgt, Cb[t]);
        T[t] = test;
        last[t] = start + j - rg.x + 1;
        if (STATS) ++n_blend;
      }
    }
  }
  if (inside) {
#pragma unroll
    for (int t = 0; t < TG; ++t) {
      if (t >= ntg) break;
      const int64_t o = (((int64_t)view * A.n_tf + t0 + t) * A.height + py) * A.width + px;
      out[o] = make_float4(add(Cr[t], mul(T[t], A.bg0)), add(Cg[t], mul(T[t], A.bg1)),
                           add(Cb[t], mul(T[t], A.bg2)), T[t]);
      n_contrib[o] = last[t];
    }
  }
  if (STATS) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n_vis += __shfl_down_sync(0xffffffffu, n_vis, o);
      n_alpha += __shfl_down_sync(0xffffffffu, n_alpha, o);
      n_blend += __shfl_down_sync(0xffffffffu, n_blend, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&stats[0], n_vis);
      atomicAdd(&stats[1], n_alpha);
      atomicAdd(&stats[2], n_blend);
    }
  }
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------

__device__ __forceinline__ void red_add_v4(float4* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
               "f"(d)
               : "memory");
}

// Replays each pixel's forward blend front to back.  With S_i the running
// sum of (c_j . g) alpha_j T_j over blended j <= i and K = C_final . g +
// T_final (bg . g + g_T), the gradient of the loss w.r.t. alpha_i is
//   dL/dalpha_i = T_i (c_i . g) - (K - S_i) / (1 - alpha_i),
// i.e. the prefix form of the suffix sum over later splats (no division
// chain to recover T).  Per splat, the seven screen-space gradients are
// reduced over the warp, summed over warps in shared memory and added to
// the per-record gradient buffer once per tile.
template <int TG, bool STATS>
__global__ void __launch_bounds__(256)
    composite_bwd_kernel(CompArgs A, const float4* __restrict__ out,
                         const int32_t* __restrict__ n_contrib, const float4* __restrict__ dout,
                         float4* __restrict__ grad2d, unsigned long long* __restrict__ stats) {
  // work counters (instrumented build only): replayed pairs, alpha
  // evaluations, blended pairs, blended pairs below the clamp, pairs with a
  // screen-space gradient
  unsigned long long n_rep = 0, n_alpha = 0, n_blend = 0, n_free = 0, n_grad = 0;
  extern __shared__ float4 smem[];
  float4* s_lut = smem;                                   // [TG][L]
  float4* s_col = s_lut + TG * A.lut_size;                // [TG][kBatch]: rgb, A w
  float4* s_slope = s_col + TG * kBatch;                  // [TG][kBatch]: drgb/dv, w dA/dv
  float4* s_geo = s_slope + TG * kBatch;                  // [kBatch]: u, -a/2, -b
  float* s_A = reinterpret_cast<float*>(s_geo + kBatch);  // [TG][kBatch]: A
  float* s_c = s_A + TG * kBatch;                         // [kBatch]: -c/2
  float* s_acc = s_c + kBatch;                            // [8][kBatch]
  uint32_t* s_idx = reinterpret_cast<uint32_t*>(s_acc + 8 * kBatch);
  __shared__ int s_maxnc;

  const int tile = blockIdx.x, view = blockIdx.y, t0 = blockIdx.z * TG;
  const int ntg = min(TG, A.n_tf - t0);
  const int L = A.lut_size;
  stage_luts<TG>(A, t0, s_lut);
  for (int e = threadIdx.x; e < 8 * kBatch; e += 256) s_acc[e] = 0.0f;
  if (threadIdx.x == 0) s_maxnc = 0;
  int px, py;
  pixel_of(tile, A.tiles_x, px, py);
  const bool inside = px < A.width && py < A.height;
  const float fx = (float)px, fy = (float)py;
  const int2 rg = A.ranges[(int64_t)view * A.tiles_per_view + tile];

  float T[TG], S[TG], K[TG], gr[TG], gg[TG], gb[TG];
  int nc[TG];
  int my_max = 0;
#pragma unroll
  for (int t = 0; t < TG; ++t) {
    T[t] = 1.0f;
    S[t] = 0.0f;
    K[t] = 0.0f;
    gr[t] = gg[t] = gb[t] = 0.0f;
    nc[t] = 0;
    if (inside && t < ntg) {
      const int64_t o = (((int64_t)view * A.n_tf + t0 + t) * A.height + py) * A.width + px;
      const float4 ov = out[o], dv4 = dout[o];
      nc[t] = n_contrib[o];
      gr[t] = dv4.x;
      gg[t] = dv4.y;
      gb[t] = dv4.z;
      const float Tn = ov.w;
      const float cr = ov.x - Tn * A.bg0, cg = ov.y - Tn * A.bg1, cb = ov.z - Tn * A.bg2;
      K[t] = cr * dv4.x + cg * dv4.y + cb * dv4.z +
             Tn * (A.bg0 * dv4.x + A.bg1 * dv4.y + A.bg2 * dv4.z + dv4.w);
      my_max = max(my_max, nc[t]);
    }
  }
  // loop bounds: a warp walks until its last pixel is done (all lanes take
  // part in the reductions); the block stages until its last warp is done
  int warp_max = my_max;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) warp_max = max(warp_max, __shfl_xor_sync(0xffffffffu, warp_max, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) atomicMax(&s_maxnc, warp_max);
  __syncthreads();
  const int block_max = s_maxnc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  for (int start = rg.x; start < rg.x + block_max; start += kBatch) {
    const int i = start + threadIdx.x;
    if (i < rg.y) {
      const uint32_t g = A.vals[i];
      const float4 ge = A.geo[g], au = A.aux[g];
      s_idx[threadIdx.x] = g;
      s_geo[threadIdx.x] = make_float4(ge.x, ge.y, -0.5f * au.x, -au.y);
      s_c[threadIdx.x] = -0.5f * au.z;
      const TfPos q = tf_pos(au.w, L);
      const bool in01 = au.w >= 0.0f && au.w <= 1.0f;
      const float sl = in01 ? (float)(L - 1) : 0.0f;
#pragma unroll
      for (int t = 0; t < TG; ++t) {
        const float4 lo = s_lut[t * L + q.k], hi = s_lut[t * L + q.k + 1];
        const float Aop = lerp_rn(lo.w, hi.w, q);
        s_col[t * kBatch + threadIdx.x] =
            make_float4(lerp_rn(lo.x, hi.x, q), lerp_rn(lo.y, hi.y, q), lerp_rn(lo.z, hi.z, q),
                        mul(Aop, ge.w));
        s_slope[t * kBatch + threadIdx.x] = make_float4(
            sl * (hi.x - lo.x), sl * (hi.y - lo.y), sl * (hi.z - lo.z), ge.w * sl * (hi.w - lo.w));
        s_A[t * kBatch + threadIdx.x] = Aop;
      }
    }
    __syncthreads();
    const int cnt = min(min(kBatch, rg.y - start), rg.x + warp_max - start);
    for (int j = 0; j < cnt; ++j) {
      const int idx = start + j - rg.x;  // list position
      float dG = 0.f, dvv = 0.f, dww = 0.f;
      const float4 sg = s_geo[j];
      const float sc = s_c[j];
      const float dx = sub(sg.x, fx), dy = sub(sg.y, fy);
      const float power = power_of(dx, dy, sg.z, sg.w, sc);
      float G = 0.f;
      if (STATS && idx < my_max) ++n_rep;
      if (idx < my_max && power <= 0.0f) {
        G = gauss_of(power);
#pragma unroll
        for (int t = 0; t < TG; ++t) {
          if (idx >= nc[t]) continue;
          if (STATS) ++n_alpha;
          const float4 c = s_col[t * kBatch + j];
          const float raw = mul(c.w, G);
          const float alpha = fminf(kAlphaMax, raw);
          if (alpha < kAlphaMin) continue;
          if (STATS) {
            ++n_blend;
            n_free += (raw <= kAlphaMax);
          }
          const float wgt = mul(alpha, T[t]);
          const float cgd = c.x * gr[t] + c.y * gg[t] + c.z * gb[t];
          S[t] += cgd * wgt;
          const float one_m = sub(1.0f, alpha);
          const float dalpha = T[t] * cgd - __fdividef(K[t] - S[t], one_m);
          const float4 sl = s_slope[t * kBatch + j];
          dvv += wgt * (gr[t] * sl.x + gg[t] * sl.y + gb[t] * sl.z);
          if (raw <= kAlphaMax) {
            const float daw = dalpha * G;
            dvv += daw * sl.w;
            dww += daw * s_A[t * kBatch + j];
            dG += dalpha * c.w;
          }
          T[t] = mul(T[t], one_m);
        }
      }
      const float dp = dG * G;
      if (STATS) n_grad += (dG != 0.f);
      float v0 = dp * (2.0f * sg.z * dx + sg.w * dy);
      float v1 = dp * (2.0f * sc * dy + sg.w * dx);
      float v2 = dp * (-0.5f * dx * dx);
      float v3 = dp * (-dx * dy);
      float v4 = dp * (-0.5f * dy * dy);
      float v5 = dvv, v6 = dww;
      const bool nz = (dp != 0.f) || (dvv != 0.f) || (dww != 0.f);
      if (__any_sync(0xffffffffu, nz)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          v0 += __shfl_xor_sync(0xffffffffu, v0, o);
          v1 += __shfl_xor_sync(0xffffffffu, v1, o);
          v2 += __shfl_xor_sync(0xffffffffu, v2, o);
          v3 += __shfl_xor_sync(0xffffffffu, v3, o);
          v4 += __shfl_xor_sync(0xffffffffu, v4, o);
          v5 += __shfl_xor_sync(0xffffffffu, v5, o);
          v6 += __shfl_xor_sync(0xffffffffu, v6, o);
        }
        if (lane == 0) {
          atomicAdd(&s_acc[0 * kBatch + j], v0);
          atomicAdd(&s_acc[1 * kBatch + j], v1);
          atomicAdd(&s_acc[2 * kBatch + j], v2);
          atomicAdd(&s_acc[3 * kBatch + j], v3);
          atomicAdd(&s_acc[4 * kBatch + j], v4);
          atomicAdd(&s_acc[5 * kBatch + j], v5);
          atomicAdd(&s_acc[6 * kBatch + j], v6);
        }
      }
    }
    (void)warp;
    __syncthreads();
    if (i < rg.y) {
      float a[7];
      bool any = false;
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        a[k] = s_acc[k * kBatch + threadIdx.x];
        s_acc[k * kBatch + threadIdx.x] = 0.0f;
        any |= (a[k] != 0.0f);
      }
      if (any) {
        float4* dst = grad2d + 2 * (int64_t)s_idx[threadIdx.x];
        red_add_v4(dst, a[0], a[1], a[2], a[3]);
        red_add_v4(dst + 1, a[4], a[5], a[6], 0.0f);
      }
    }
    __syncthreads();
  }
  if (STATS) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n_rep += __shfl_down_sync(0xffffffffu, n_rep, o);
      n_alpha += __shfl_down_sync(0xffffffffu, n_alpha, o);
      n_blend += __shfl_down_sync(0xffffffffu, n_blend, o);
      n_free += __shfl_down_sync(0xffffffffu, n_free, o);
      n_grad += __shfl_down_sync(0xffffffffu, n_grad, o);
    }
    if (lane == 0) {
      atomicAdd(&stats[0], n_rep);
      atomicAdd(&stats[1], n_alpha);
      atomicAdd(&stats[2], n_blend);
      atomicAdd(&stats[3], n_free);
      atomicAdd(&stats[4], n_grad);
    }
  }
}

size_t bwd_smem_bytes(int TG, int L) {
  return (size_t)TG * L * 16 + (size_t)TG * kBatch * 16 * 2 + (size_t)kBatch * 16 +
         (size_t)TG * kBatch * 4 + (size_t)kBatch * 4 + (size_t)8 * kBatch * 4 +
         (size_t)kBatch * 4;
}

int pick_group(int tf_group, int n_tf, bool bwd) {
  int g = tf_group;
  if (g <= 0) g = std::min(n_tf, 4);
  if (g <= 1) return 1;
  if (g <= 2) return 2;
  if (g <= 4 || bwd) return 4;
  return 8;
}

CompArgs make_args(const veg_camera* cams, int64_t n, const float4* geo, const float4* aux,
                   const uint32_t* vals, const int2* ranges, veg_tf tf, const float* bg) {
  CompArgs A;
  A.geo = geo;
  A.aux = aux;
  A.vals = vals;
  A.ranges = ranges;
  A.lut = reinterpret_cast<const float4*>(tf.lut);
  A.lut_size = tf.lut_size;
  A.n_tf = tf.n_tf;
  A.width = cams[0].width;
  A.height = cams[0].height;
  A.tiles_x = tiles_x_of(A.width);
  A.tiles_per_view = A.tiles_x * tiles_x_of(A.height);
  A.bg0 = bg ? bg[0] : 0.f;
  A.bg1 = bg ? bg[1] : 0.f;
  A.bg2 = bg ? bg[2] : 0.f;
  (void)n;
  return A;
}

// Allows `dyn` bytes of dynamic shared memory for `kern` (once per size
// increase); refuses sizes beyond the 227 KB a CTA may hold.
template <typename K>
veg_status prepare_smem(K kern, size_t dyn, size_t* configured) {
  if (dyn <= *configured) return VEG_OK;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return VEG_ERR_CUDA;
  if (fa.sharedSizeBytes + dyn > 227 * 1024) return VEG_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) !=
      cudaSuccess)
    return VEG_ERR_UNSUPPORTED;
  *configured = dyn;
  return VEG_OK;
}

template <int TG, bool STATS>
veg_status launch_fwd_t(const CompArgs& A, int n_views, float4* out, int32_t* nc,
                        unsigned long long* stats, cudaStream_t stream) {
  const size_t smem = (size_t)TG * A.lut_size * sizeof(float4);
  auto kern = composite_fwd_kernel<TG, STATS>;
  static size_t configured = 0;
  veg_status st = prepare_smem(kern, smem, &configured);
  if (st != VEG_OK) return st;
  dim3 grid((unsigned)A.tiles_per_view, (unsigned)n_views, (unsigned)((A.n_tf + TG - 1) / TG));
  kern<<<grid, 256, smem, stream>>>(A, out, nc, stats);
  count_launch();
  return launch_status();
}

template <int TG, bool STATS>
veg_status launch_bwd_t(const CompArgs& A, int n_views, const float4* out, const int32_t* nc,
                        const float4* dout, float4* grad2d, unsigned long long* stats,
                        cudaStream_t stream) {
  const size_t smem = bwd_smem_bytes(TG, A.lut_size);
  auto kern = composite_bwd_kernel<TG, STATS>;
  static size_t configured = 0;
  veg_status st = prepare_smem(kern, smem, &configured);
  if (st != VEG_OK) return st;
  dim3 grid((unsigned)A.tiles_per_view, (unsigned)n_views, (unsigned)((A.n_tf + TG - 1) / TG));
  kern<<<grid, 256, smem, stream>>>(A, out, nc, dout, grad2d, stats);
  count_launch();
  return launch_status();
}

}  // namespace

veg_status project_bwd_launch(const CamSet& cs, int n_views, veg_gaussians g,
                              const int32_t* tiles, const float4* grad2d, float4* gm, float4* gl,
                              float4* gq, cudaStream_t stream);

veg_status composite_fwd_launch(const veg_camera* cams, int n_views, int64_t n,
                                const float4* geo, const float4* aux, const uint32_t* vals,
                                const int2* ranges, veg_tf tf, const float* bg, int tf_group,
                                float4* out, int32_t* n_contrib, unsigned long long* stats,
                                cudaStream_t stream) {
  CompArgs A = make_args(cams, n, geo, aux, vals, ranges, tf, bg);
  const int TG = pick_group(tf_group, tf.n_tf, false);
  if (stats) {
    switch (TG) {
      case 1: return launch_fwd_t<1, true>(A, n_views, out, n_contrib, stats, stream);
      case 2: return launch_fwd_t<2, true>(A, n_views, out, n_contrib, stats, stream);
      case 4: return launch_fwd_t<4, true>(A, n_views, out, n_contrib, stats, stream);
      default: return launch_fwd_t<8, true>(A, n_views, out, n_contrib, stats, stream);
    }
  }
  switch (TG) {
    case 1: return launch_fwd_t<1, false>(A, n_views, out, n_contrib, nullptr, stream);
    case 2: return launch_fwd_t<2, false>(A, n_views, out, n_contrib, nullptr, stream);
    case 4: return launch_fwd_t<4, false>(A, n_views, out, n_contrib, nullptr, stream);
    default: return launch_fwd_t<8, false>(A, n_views, out, n_contrib, nullptr, stream);
  }
}

size_t composite_bwd_ws_bytes(int64_t n, int n_views) {
  Carver c(nullptr);
  c.take<float4>((size_t)2 * n * n_views);
  return c.bytes();
}

}  // namespace veg

using namespace veg;

static veg_status check_composite_common(const veg_camera* cams, int32_t n_views, int64_t n,
                                         const float* geo, const float* aux, const uint32_t* vals,
                                         const int32_t* ranges, veg_tf tf) {
  veg_status st = check_cameras(cams, n_views);
  if (st != VEG_OK) return st;
  if (n < 0 || !ranges || !tf.lut || tf.lut_size < 2 || tf.n_tf < 1 || tf.n_tf > 4096)
    return VEG_ERR_INVALID_ARGUMENT;
  if (tf.lut_size > 4096) return VEG_ERR_UNSUPPORTED;
  if (n > 0 && (!geo || !aux || !vals)) return VEG_ERR_INVALID_ARGUMENT;
  if (!aligned16(geo) || !aligned16(aux) || !aligned16(tf.lut) ||
      (reinterpret_cast<uintptr_t>(ranges) & 7))
    return VEG_ERR_INVALID_ARGUMENT;
  return VEG_OK;
}

extern "C" veg_status veg_composite_fwd(const veg_camera* cams, int32_t n_views, int64_t n,
                                        const float* splat_geo, const float* splat_aux,
                                        const uint32_t* vals, const int32_t* tile_ranges,
                                        veg_tf tf, const float* bg, int32_t tf_group, float* out,
                                        int32_t* n_contrib, unsigned long long* stats,
                                        cudaStream_t stream) {
  veg_status st =
      check_composite_common(cams, n_views, n, splat_geo, splat_aux, vals, tile_ranges, tf);
  if (st != VEG_OK) return st;
  if (!out || !n_contrib || !aligned16(out) || tf_group < 0 || tf_group > 8)
    return VEG_ERR_INVALID_ARGUMENT;
  return composite_fwd_launch(cams, n_views, n, reinterpret_cast<const float4*>(splat_geo),
                              reinterpret_cast<const float4*>(splat_aux), vals,
                              reinterpret_cast<const int2*>(tile_ranges), tf, bg, tf_group,
                              reinterpret_cast<float4*>(out), n_contrib, stats, stream);
}

extern "C" veg_status veg_composite_bwd_workspace_size(int64_t n, int32_t n_views,
                                                       size_t* bytes) {
  if (!bytes || n < 0 || n_views < 1 || n_views > VEG_MAX_VIEWS) return VEG_ERR_INVALID_ARGUMENT;
  *bytes = composite_bwd_ws_bytes(n, n_views);
  return VEG_OK;
}

extern "C" veg_status veg_composite_bwd(const veg_camera* cams, int32_t n_views, veg_gaussians g,
                                        const float* splat_geo, const float* splat_aux,
                                        const int32_t* tiles_touched, const uint32_t* vals,
                                        const int32_t* tile_ranges, veg_tf tf, const float* bg,
                                        int32_t tf_group, const float* out,
                                        const int32_t* n_contrib, const float* dL_dout,
                                        void* workspace, size_t workspace_bytes,
                                        float* grad_mean_v, float* grad_logscale_w,
                                        float* grad_quat, float* grad2d,
                                        unsigned long long* stats, cudaStream_t stream) {
  veg_status st =
      check_composite_common(cams, n_views, g.n, splat_geo, splat_aux, vals, tile_ranges, tf);
  if (st != VEG_OK) return st;
  if (!out || !n_contrib || !dL_dout || !aligned16(out) || !aligned16(dL_dout) || tf_group < 0 ||
      tf_group > 8)
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
  CompArgs A = make_args(cams, g.n, reinterpret_cast<const float4*>(splat_geo),
                         reinterpret_cast<const float4*>(splat_aux), vals,
                         reinterpret_cast<const int2*>(tile_ranges), tf, bg);
  const int TG = pick_group(tf_group, tf.n_tf, true);
  const float4* o4 = reinterpret_cast<const float4*>(out);
  const float4* d4 = reinterpret_cast<const float4*>(dL_dout);
  if (stats) {
    switch (TG) {
      case 1: st = launch_bwd_t<1, true>(A, n_views, o4, n_contrib, d4, g2, stats, stream); break;
      case 2: st = launch_bwd_t<2, true>(A, n_views, o4, n_contrib, d4, g2, stats, stream); break;
      default: st = launch_bwd_t<4, true>(A, n_views, o4, n_contrib, d4, g2, stats, stream); break;
    }
  } else {
    switch (TG) {
      case 1: st = launch_bwd_t<1, false>(A, n_views, o4, n_contrib, d4, g2, nullptr, stream); break;
      case 2: st = launch_bwd_t<2, false>(A, n_views, o4, n_contrib, d4, g2, nullptr, stream); break;
      default: st = launch_bwd_t<4, false>(A, n_views, o4, n_contrib, d4, g2, nullptr, stream); break;
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

extern "C" veg_status veg_project_bwd(const veg_camera* cams, int32_t n_views, veg_gaussians g,
                                      const int32_t* tiles_touched, const float* grad2d,
                                      float* grad_mean_v, float* grad_logscale_w,
                                      float* grad_quat, cudaStream_t stream) {
  veg_status st = check_cameras(cams, n_views);
  if (st != VEG_OK) return st;
  if (g.n < 0 || g.n * n_views >= ((int64_t)1 << 31)) return VEG_ERR_INVALID_ARGUMENT;
  if (g.n > 0 && (!g.mean_v || !g.logscale_w || !g.quat || !tiles_touched || !grad2d ||
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
                            reinterpret_cast<float4*>(grad_quat), stream);
}
