// Emission-absorption raymarching of a gridded scalar volume: the renderer
// of the paper's training images (Sec. 4.2, 5.1: the volume is raymarched
// with an emission-absorption model and shaded with Blinn-Phong lighting
// from a headlight).
//
// Volume: R^3 vertices on [-1,1]^3 (x fastest), prepared once as float4
// (value, d/dx, d/dy, d/dz) with central-difference vertex gradients
// (one-sided on the boundary), so one sample is eight float4 loads and a
// trilinear blend of value and gradient together.
//
// Per ray (one thread per pixel, 16 x 16 pixels per CTA): the camera ray is
// clipped to the box and to the near plane; samples sit at t0 + (k + 1/2)
// Delta; each sample's transfer-function colour and opacity (tables of the
// CTA's group in shared memory) give alpha = 1 - (1 - A)^(Delta / h), the
// colour is Blinn-Phong shaded with the interpolated gradient (ambient only
// where it vanishes), and the
// samples are composited front to back until every table of the group has
// T < 1e-4.
#include <algorithm>
#include <cmath>

#include "veg_internal.cuh"

namespace veg {

namespace {

// Hardware approximations of 2^x and log2 x (the opacity correction), whose
// errors stay far below the image tolerance.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct RayView {
  float r[9];      // world-to-camera rotation, row-major
  float eye[3];    // camera centre
  float light[3];  // headlight direction (toward the light)
  float fx, fy, cx, cy, near_plane;
};

struct RaySet {
  RayView v[VEG_MAX_VIEWS];
};

struct MarchArgs {
  const float4* vol;
  int R;
  float inv_h, step, ratio;  // ratio = step / h
  const float4* lut;
  int lut_size, n_tf;
  const int32_t* view_tf;
  int width, height, tiles_x, tiles_per_view;
  bool shade;
  float ka, kd, ks, beta;
  float bg0, bg1, bg2;
  // empty-space skipping: per-macrocell table masks (veg_raymarch_cells)
  // over macrocells of 2^cell_shift vertex cells per axis, or null
  const uint32_t* cell_mask;
  int cell_shift, cells;
};

__global__ void __launch_bounds__(256)
    volume_prepare_kernel(const float* __restrict__ vol, int R, float inv_h, float4* __restrict__ out) {
  pdl_enter();
  const int64_t n = (int64_t)R * R * R;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int x = (int)(i % R), y = (int)((i / R) % R), z = (int)(i / ((int64_t)R * R));
  const int64_t sx = 1, sy = R, sz = (int64_t)R * R;
  auto diff = [&](int c, int64_t s) {
    if (c == 0) return (vol[i + s] - vol[i]) * inv_h;
    if (c == R - 1) return (vol[i] - vol[i - s]) * inv_h;
    return (vol[i + s] - vol[i - s]) * (0.5f * inv_h);
  };
  out[i] = make_float4(vol[i], diff(x, sx), diff(y, sy), diff(z, sz));
}

// Per macrocell (cell^3 vertex cells, vertices [c cell, c cell + cell] per
// axis clipped to the grid): bit t (t < 32) set when table t can give a
// sample in the cell a nonzero opacity.  A sample's value is a trilinear
// blend of the cell's vertex values, so it lies in their [min, max] up to
// rounding; the test widens the range by 1e-6 and takes the table entries
// that values in it interpolate between, with one more entry on each side,
// and sets the bit when any of them has a positive opacity (interpolating
// two non-positive entries gives a clamped opacity of 0).  A NaN vertex, or
// more than 32 tables, sets every bit.
__global__ void __launch_bounds__(256)
    cell_mask_kernel(const float4* __restrict__ vol, int R, int cell, int cells,
                     const float4* __restrict__ lut, int L, int n_tf, uint32_t* __restrict__ mask) {
  pdl_enter();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nc = (int64_t)cells * cells * cells;
  if (i >= nc) return;
  const int cx = (int)(i % cells), cy = (int)((i / cells) % cells), cz = (int)(i / ((int64_t)cells * cells));
  const int x0 = cx * cell, y0 = cy * cell, z0 = cz * cell;
  const int x1 = min(x0 + cell, R - 1), y1 = min(y0 + cell, R - 1), z1 = min(z0 + cell, R - 1);
  float mn = 3.0e38f, mx = -3.0e38f;
  bool nan = false;
  for (int z = z0; z <= z1; ++z)
    for (int y = y0; y <= y1; ++y)
      for (int x = x0; x <= x1; ++x) {
        const float v = __ldg(&vol[((int64_t)z * R + y) * R + x]).x;
        nan |= v != v;
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
      }
  uint32_t m = 0u;
  if (nan || n_tf > 32) {
    m = 0xffffffffu;
  } else {
    const float lo = fminf(fmaxf(mn - 1e-6f, 0.0f), 1.0f) * (float)(L - 1);
    const float hi = fminf(fmaxf(mx + 1e-6f, 0.0f), 1.0f) * (float)(L - 1);
    const int k0 = max((int)floorf(lo) - 1, 0), k1 = min((int)floorf(hi) + 2, L - 1);
    for (int t = 0; t < n_tf; ++t)
      for (int k = k0; k <= k1; ++k)
        if (__ldg(&lut[(int64_t)t * L + k]).w > 0.0f) {
          m |= 1u << t;
          break;
        }
  }
  mask[i] = m;
}

// stats (instrumented build): samples taken (per ray and table group),
// table evaluations (samples x live tables) and, with a cell mask, samples
// skipped as empty.
template <int TG, bool STATS>
__global__ void __launch_bounds__(256)
    raymarch_kernel(MarchArgs A, RaySet rs, float4* __restrict__ out,
                    unsigned long long* __restrict__ stats) {
  pdl_enter();
  unsigned long long n_samp = 0, n_tab = 0, n_skip = 0;
  extern __shared__ float4 s_lut[];
  const int wi = blockIdx.x;
  const int view = wi / A.tiles_per_view, tile = wi - view * A.tiles_per_view;
  const int t0g = blockIdx.z * TG;
  const int lut0 = A.view_tf ? A.view_tf[view] : t0g;
  const int ntg = A.view_tf ? 1 : min(TG, A.n_tf - t0g);
  const int n_out = A.view_tf ? 1 : A.n_tf;
  const int L = A.lut_size;
  for (int e = threadIdx.x; e < TG * L; e += blockDim.x) {
    const int t = e / L, k = e - t * L, ti = lut0 + t;
    s_lut[e] = (t < ntg && ti >= 0 && ti < A.n_tf) ? __ldg(&A.lut[(int64_t)ti * L + k])
                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  const int px = (tile % A.tiles_x) * VEG_TILE + (threadIdx.x & 15);
  const int py = (tile / A.tiles_x) * VEG_TILE + (threadIdx.x >> 4);
  const bool inside = px < A.width && py < A.height;
  if (!STATS && !inside) return;
  if (inside) {
  const RayView& V = rs.v[view];
  // ray direction R^T ((px - cx)/fx, (py - cy)/fy, 1), normalised
  const float ux = (px - V.cx) / V.fx, uy = (py - V.cy) / V.fy;
  float d[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) d[c] = V.r[c] * ux + V.r[3 + c] * uy + V.r[6 + c];
  const float inv_len = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
  for (int c = 0; c < 3; ++c) d[c] *= inv_len;
  // slab clip against [-1,1]^3 and t >= near
  float ta = V.near_plane, tb = 3.0e38f;
  bool hit = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (d[c] == 0.0f) {
      if (fabsf(V.eye[c]) > 1.0f) hit = false;
      continue;
    }
    const float inv = 1.0f / d[c];
    const float t1 = (-1.0f - V.eye[c]) * inv, t2 = (1.0f - V.eye[c]) * inv;
    ta = fmaxf(ta, fminf(t1, t2));
    tb = fminf(tb, fmaxf(t1, t2));
  }
  float T[TG], Cr[TG], Cg[TG], Cb[TG];
#pragma unroll
  for (int t = 0; t < TG; ++t) {
    T[t] = 1.0f;
    Cr[t] = Cg[t] = Cb[t] = 0.0f;
  }
  unsigned live = (1u << ntg) - 1u;
  if (hit && tb > ta) {
    const int n = (int)floorf((tb - ta) / A.step);
    // half vector of the view direction e = -d and the headlight
    float hv[3];
    float hn = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      hv[c] = V.light[c] - d[c];
      hn += hv[c] * hv[c];
    }
    hn = hn > 0.f ? rsqrtf(hn) : 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) hv[c] *= hn;
    const int R = A.R;
    // the group's tables occupy bits lut0 .. lut0 + ntg - 1 of a cell mask
    const bool skip_empty = A.cell_mask != nullptr && lut0 >= 0 && lut0 + ntg <= 32;
    for (int k = 0; k < n && live; ++k) {
      const float t = fmaf((float)k + 0.5f, A.step, ta);
      float g[3];
      int ic[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        g[c] = (fmaf(t, d[c], V.eye[c]) + 1.0f) * A.inv_h;
        ic[c] = min(max((int)floorf(g[c]), 0), R - 2);
        g[c] -= (float)ic[c];
      }
      if (skip_empty) {
        // every table still compositing has zero opacity in this macrocell:
        // the sample would leave colour and transmittance unchanged
        const int mc = ((ic[2] >> A.cell_shift) * A.cells + (ic[1] >> A.cell_shift)) * A.cells +
                       (ic[0] >> A.cell_shift);
        if (((__ldg(&A.cell_mask[mc]) >> lut0) & live) == 0u) {
          if (STATS) ++n_skip;
          continue;
        }
      }
      const float4* base = A.vol + ((int64_t)ic[2] * R + ic[1]) * R + ic[0];
      const int64_t sy = R, sz = (int64_t)R * R;
      auto lerp4 = [](float4 a, float4 b, float f) {
        return make_float4(fmaf(f, b.x - a.x, a.x), fmaf(f, b.y - a.y, a.y),
                           fmaf(f, b.z - a.z, a.z), fmaf(f, b.w - a.w, a.w));
      };
      const float4 c00 = lerp4(__ldg(base), __ldg(base + 1), g[0]);
      const float4 c01 = lerp4(__ldg(base + sy), __ldg(base + sy + 1), g[0]);
      const float4 c10 = lerp4(__ldg(base + sz), __ldg(base + sz + 1), g[0]);
      const float4 c11 = lerp4(__ldg(base + sz + sy), __ldg(base + sz + sy + 1), g[0]);
      const float4 s = lerp4(lerp4(c00, c01, g[1]), lerp4(c10, c11, g[1]), g[2]);
      float sd = 1.0f, ss = 0.0f;
      if (A.shade) {
        // normal = -gradient / |gradient|; scaled by the largest component
        // first so that tiny gradients cannot underflow
        const float m = fmaxf(fmaxf(fabsf(s.y), fabsf(s.z)), fabsf(s.w));
        sd = A.ka;
        if (m > 0.0f) {
          const float gx = s.y / m, gy = s.z / m, gz = s.w / m;
          const float ig = rsqrtf(gx * gx + gy * gy + gz * gz);
          const float nl = fabsf((gx * V.light[0] + gy * V.light[1] + gz * V.light[2]) * ig);
          const float nh = fabsf((gx * hv[0] + gy * hv[1] + gz * hv[2]) * ig);
          sd = A.ka + A.kd * nl;
          ss = nl > 0.f ? A.ks * __powf(nh, A.beta) : 0.f;
        }
      }
      const TfPos q = tf_pos(s.x, L);
      if (STATS) {
        ++n_samp;
        n_tab += (unsigned)__popc(live);
      }
#pragma unroll
      for (int tt = 0; tt < TG; ++tt) {
        if (!(live & (1u << tt))) continue;
        const float4 lo = s_lut[tt * L + q.k], hi = s_lut[tt * L + q.k + 1];
        const float a = fminf(fmaxf(lerp_rn(lo.w, hi.w, q), 0.0f), 1.0f);
        const float alpha = a > 0.0f ? 1.0f - ex2_approx(lg2_approx(1.0f - a) * A.ratio) : 0.0f;
        const float w = T[tt] * alpha;
        Cr[tt] = fmaf(w, fmaf(sd, lerp_rn(lo.x, hi.x, q), ss), Cr[tt]);
        Cg[tt] = fmaf(w, fmaf(sd, lerp_rn(lo.y, hi.y, q), ss), Cg[tt]);
        Cb[tt] = fmaf(w, fmaf(sd, lerp_rn(lo.z, hi.z, q), ss), Cb[tt]);
        T[tt] *= 1.0f - alpha;
        if (T[tt] < kTMin) live &= ~(1u << tt);
      }
    }
  }
#pragma unroll
  for (int tt = 0; tt < TG; ++tt) {
    if (tt >= ntg) break;
    const int64_t o = (((int64_t)view * n_out + t0g + tt) * A.height + py) * A.width + px;
    out[o] = make_float4(fmaf(T[tt], A.bg0, Cr[tt]), fmaf(T[tt], A.bg1, Cg[tt]),
                         fmaf(T[tt], A.bg2, Cb[tt]), T[tt]);
  }
  }
  if (STATS) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n_samp += __shfl_down_sync(0xffffffffu, n_samp, o);
      n_tab += __shfl_down_sync(0xffffffffu, n_tab, o);
      n_skip += __shfl_down_sync(0xffffffffu, n_skip, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&stats[0], n_samp);
      atomicAdd(&stats[1], n_tab);
      if (A.cell_mask) atomicAdd(&stats[2], n_skip);
    }
  }
}

template <int TG, bool STATS>
veg_status launch_march(const MarchArgs& A, const RaySet& rs, int n_views, float4* out,
                        unsigned long long* stats, cudaStream_t stream) {
  const size_t smem = (size_t)TG * A.lut_size * sizeof(float4);
  static SmemRecord configured;  // default carveout: the volume samples want L1
  veg_status st = prepare_smem(raymarch_kernel<TG, STATS>, smem, configured, false);
  if (st != VEG_OK) return st;
  const unsigned groups = A.view_tf ? 1u : (unsigned)((A.n_tf + TG - 1) / TG);
  dim3 grid((unsigned)(A.tiles_per_view * n_views), 1u, groups);
  launch_k(raymarch_kernel<TG, STATS>, grid, 256, smem, stream, A, rs, out, stats);
  count_launch();
  return launch_status();
}

template <int TG>
veg_status launch_march_s(const MarchArgs& A, const RaySet& rs, int n_views, float4* out,
                          unsigned long long* stats, cudaStream_t stream) {
  return stats ? launch_march<TG, true>(A, rs, n_views, out, stats, stream)
               : launch_march<TG, false>(A, rs, n_views, out, nullptr, stream);
}

}  // namespace

}  // namespace veg

using namespace veg;

extern "C" veg_status veg_volume_prepare(const float* volume, int32_t resolution, float* vol4,
                                         cudaStream_t stream) {
  if (!volume || !vol4 || resolution < 2 || resolution > 2048 || !aligned16(vol4))
    return VEG_ERR_INVALID_ARGUMENT;
  const int64_t n = (int64_t)resolution * resolution * resolution;
  const float inv_h = (float)((resolution - 1) / 2.0);
  launch_k(volume_prepare_kernel, (unsigned)((n + 255) / 256), 256, 0, stream, 
      volume, resolution, inv_h, reinterpret_cast<float4*>(vol4));
  count_launch();
  return launch_status();
}

namespace {

bool cell_size_ok(int32_t cell) { return cell >= 1 && cell <= 64 && (cell & (cell - 1)) == 0; }

int cells_per_axis(int32_t resolution, int32_t cell) {
  return (resolution - 1 + cell - 1) / cell;  // macrocells covering the R - 1 vertex cells
}

}  // namespace

extern "C" veg_status veg_raymarch_cells_count(int32_t resolution, int32_t cell, int64_t* count) {
  if (!count || resolution < 2 || resolution > 2048 || !cell_size_ok(cell))
    return VEG_ERR_INVALID_ARGUMENT;
  const int64_t c = cells_per_axis(resolution, cell);
  *count = c * c * c;
  return VEG_OK;
}

extern "C" veg_status veg_raymarch_cells(const float* vol4, int32_t resolution, veg_tf tf,
                                         int32_t cell, uint32_t* mask, cudaStream_t stream) {
  if (!vol4 || !mask || resolution < 2 || resolution > 2048 || !cell_size_ok(cell) || !tf.lut ||
      tf.lut_size < 2 || tf.n_tf < 1 || !aligned16(vol4) || !aligned16(tf.lut))
    return VEG_ERR_INVALID_ARGUMENT;
  const int c = cells_per_axis(resolution, cell);
  const int64_t nc = (int64_t)c * c * c;
  launch_k(cell_mask_kernel, (unsigned)((nc + 255) / 256), 256, 0, stream, 
      reinterpret_cast<const float4*>(vol4), resolution, cell, c,
      reinterpret_cast<const float4*>(tf.lut), tf.lut_size, tf.n_tf, mask);
  count_launch();
  return launch_status();
}

extern "C" veg_status veg_raymarch_masked(const veg_camera* cams, int32_t n_views,
                                          const float* vol4, int32_t resolution, veg_tf tf,
                                          float step, const veg_material* material,
                                          const float* bg, const uint32_t* cell_mask,
                                          int32_t cell, float* out, unsigned long long* stats,
                                          cudaStream_t stream) {
  veg_status st = check_cameras_one_size(cams, n_views);
  if (st != VEG_OK) return st;
  if (!vol4 || !out || resolution < 2 || resolution > 2048 || !(step > 0.0f) || !tf.lut ||
      tf.lut_size < 2 || tf.n_tf < 1 || !aligned16(vol4) || !aligned16(out) ||
      !aligned16(tf.lut) || (cell_mask && !cell_size_ok(cell)))
    return VEG_ERR_INVALID_ARGUMENT;
  if (tf.lut_size > 4096) return VEG_ERR_UNSUPPORTED;
  MarchArgs A;
  A.cell_mask = cell_mask;
  A.cell_shift = 0;
  while (cell_mask && (1 << A.cell_shift) < cell) ++A.cell_shift;
  A.cells = cell_mask ? cells_per_axis(resolution, cell) : 0;
  A.vol = reinterpret_cast<const float4*>(vol4);
  A.R = resolution;
  const double h = 2.0 / (resolution - 1);
  A.inv_h = (float)(1.0 / h);
  A.step = step;
  A.ratio = (float)(step / h);
  A.lut = reinterpret_cast<const float4*>(tf.lut);
  A.lut_size = tf.lut_size;
  A.n_tf = tf.n_tf;
  A.view_tf = tf.view_tf;
  A.width = cams[0].width;
  A.height = cams[0].height;
  A.tiles_x = tiles_x_of(A.width);
  A.tiles_per_view = A.tiles_x * tiles_x_of(A.height);
  A.shade = material != nullptr;
  A.ka = material ? material->ka : 0.f;
  A.kd = material ? material->kd : 0.f;
  A.ks = material ? material->ks : 0.f;
  A.beta = material ? material->beta : 0.f;
  A.bg0 = bg ? bg[0] : 0.f;
  A.bg1 = bg ? bg[1] : 0.f;
  A.bg2 = bg ? bg[2] : 0.f;
  RaySet rs;
  for (int v = 0; v < n_views; ++v) {
    const float* w = cams[v].world_to_cam;
    RayView& V = rs.v[v];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) V.r[r * 3 + c] = w[r * 4 + c];
    for (int c = 0; c < 3; ++c) {
      V.eye[c] = -(w[0 * 4 + c] * w[3] + w[1 * 4 + c] * w[7] + w[2 * 4 + c] * w[11]);
      V.light[c] = -w[2 * 4 + c];
    }
    V.fx = cams[v].fx;
    V.fy = cams[v].fy;
    V.cx = cams[v].cx;
    V.cy = cams[v].cy;
    V.near_plane = cams[v].near_plane;
  }
  float4* o = reinterpret_cast<float4*>(out);
  // tables per sample pass: up to 8, halved until they fit a CTA's shared
  // memory (one table of up to 4096 entries always fits)
  int g = tf.view_tf ? 1 : std::min(tf.n_tf, 8);
  while (g > 1 && (size_t)g * tf.lut_size * sizeof(float4) > (size_t)227 * 1024) g /= 2;
  if (g <= 1) return launch_march_s<1>(A, rs, n_views, o, stats, stream);
  if (g <= 2) return launch_march_s<2>(A, rs, n_views, o, stats, stream);
  if (g <= 4) return launch_march_s<4>(A, rs, n_views, o, stats, stream);
  return launch_march_s<8>(A, rs, n_views, o, stats, stream);
}

extern "C" veg_status veg_raymarch(const veg_camera* cams, int32_t n_views, const float* vol4,
                                   int32_t resolution, veg_tf tf, float step,
                                   const veg_material* material, const float* bg, float* out,
                                   unsigned long long* stats, cudaStream_t stream) {
  return veg_raymarch_masked(cams, n_views, vol4, resolution, tf, step, material, bg, nullptr, 1,
                             out, stats, stream);
}
