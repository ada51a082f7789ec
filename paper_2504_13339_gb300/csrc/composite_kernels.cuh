// Compositing kernels: front-to-back blending (Eq. 1) of depth-sorted splats
// per 16x16 tile for a group of transfer functions, and its backward pass.
//
// One CTA of 256 threads owns one (view, tile, TF group) work item, in the
// longest-first order of the tiles; each thread owns one pixel and each warp
// an 8x4 pixel block.  The tile's list is staged in batches of B splats (the
// tile batch: 128, 256 or 512, chosen by the caller or its autotuner)
// through shared memory.  The stager evaluates every
// splat's colour and opacity under each TF of the group once (linear
// interpolation in the TF tables: held in shared memory by the forward, read
// through the L1 cache by the backward), the exponent below which
// no TF of the group can reach alpha = 1/255, and a conservative mask of the
// warp blocks that the splat's visible ellipse can touch.  Each warp then
// compacts the batch into its own list (ballots) and walks only that list,
// so pairs that provably cannot blend cost nothing.  A pixel leaves once
// every TF of the group has terminated (T (1 - alpha) < 1e-4); the block
// stops staging once all its pixels have left.
//
// The per-pair arithmetic that decides skips, the 0.99 clamp and
// termination uses explicitly rounded operations shared by the forward and
// backward kernels, so the backward replays every forward decision bit for
// bit.  Culling (cutoff, warp mask) only removes pairs whose alpha is
// provably below 1/255, so it never changes a decision.
#pragma once

#include <algorithm>

#include "veg_internal.cuh"

namespace veg {

namespace {

constexpr int kWarps = 8;  // 256 threads
// Every per-splat shared array is indexed by the splat's batch slot, which
// a thread loops over in steps of the block size (B / 256 slots per thread
// for B = 512; threads past the slots stage nothing for B = 128).

// A warp list entry is a batch slot: one byte for batches up to 256 splats.
template <int B>
struct ListEntry {
  using T = unsigned char;
};
template <>
struct ListEntry<512> {
  using T = unsigned short;
};

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

// The same exponent from the splat centre (ux, uy) and the pixel pxy, with
// the offsets d = u - p and their squares d2 formed as float32 pairs (same
// rounding as the scalar form); also returns dxy = dx dy.
__device__ __forceinline__ float power_at(float ux, float uy, float2 pxy, float na, float nb,
                                          float nc, float2& d, float2& d2, float& dxy) {
  d = sub2(make_float2(ux, uy), pxy);
  d2 = mul2(d, d);
  dxy = mul(d.x, d.y);
  return __fmaf_rn(na, d2.x, __fmaf_rn(nc, d2.y, mul(nb, dxy)));
}

// Lowest exponent at which some TF of the group can still reach alpha >=
// 1/255: alpha = A w G <= max_t(A_t w) e^power, which stays below 1/255 for
// power < ln(1/(255 max_t A_t w)).  The bound is lowered by 1e-3 to absorb
// the float32 rounding of the exponent, the exp2 approximation and the log,
// so every pair above it still meets the exact per-TF test and the skip
// never changes a decision.  With max_t A_t w < 1/255 no pair can blend.
__device__ __forceinline__ float power_cutoff(float max_aw) {
  if (!(max_aw >= kAlphaMin)) return 1.0f;
  return __logf(kAlphaMin) - __logf(max_aw) - 1e-3f;
}

// Hardware approximations (relative error of a few 1e-7), used only where
// a bound carries a far wider margin.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Minimum of q(d) = a dx^2 + 2 b dx dy + c dy^2 (a, c > 0, positive
// definite) over the rectangle [x0, x1] x [y0, y1]: zero when the rectangle
// holds the origin, else the least of the four edge minima (on an edge q is
// a 1-D convex quadratic, minimised at its vertex clamped to the edge).
__device__ __forceinline__ float conic_min_over_rect(float a, float b, float c, float x0,
                                                     float x1, float y0, float y1) {
  if (x0 <= 0.0f && x1 >= 0.0f && y0 <= 0.0f && y1 >= 0.0f) return 0.0f;
  auto qf = [&](float x, float y) { return a * x * x + 2.0f * b * x * y + c * y * y; };
  const float ia = rcp_approx(a), ic = rcp_approx(c);
  float m = qf(x0, fminf(fmaxf(-b * x0 * ic, y0), y1));
  m = fminf(m, qf(x1, fminf(fmaxf(-b * x1 * ic, y0), y1)));
  m = fminf(m, qf(fminf(fmaxf(-b * y0 * ia, x0), x1), y0));
  m = fminf(m, qf(fminf(fmaxf(-b * y1 * ia, x0), x1), y1));
  return m;
}

// Warp blocks (bit by*2+bx for the 8x4 block at tile-relative (8bx, 4by))
// holding a pixel centre where the exponent can reach `cut`, i.e. a centre d
// (relative to the splat centre) with d^T Q d <= -2 cut (Q = conic).  A
// block's bounding-box test rejects far blocks; the rest are kept when the
// quadratic's minimum over the block's rectangle of pixel centres is within
// the radius.  Box half extents are widened by 0.2% + 0.02 px and the
// squared radius by 0.2% + 1e-4, far beyond the float32 error of the
// per-pixel exponent, so the mask never drops a pixel the exact test keeps.
// An ill-conditioned conic keeps every block (the per-pixel test decides).
// EXACT = false keeps every block passing the box test (cheaper to stage;
// the forward pass, whose iterations are cheap, prefers it).
template <bool EXACT>
__device__ __forceinline__ unsigned warp_block_mask(float rx, float ry, float a, float b, float c,
                                                    float cut) {
  if (!(cut < 0.0f)) return 0u;
  const float det = a * c - b * b;
  if (!(det > 1e-3f * a * c)) return 0xffu;
  const float r2 = -2.0f * cut, r2_det = r2 * rcp_approx(det);
  const float hx = sqrt_approx(r2_det * c) * 1.002f + 0.02f;
  const float hy = sqrt_approx(r2_det * a) * 1.002f + 0.02f;
  const float r2m = r2 * 1.002f + 1e-4f;
  const float x0 = rx - hx, x1 = rx + hx, y0 = ry - hy, y1 = ry + hy;
  unsigned m = 0u;
#pragma unroll
  for (int by = 0; by < 4; ++by) {
    if (y1 < 4.0f * by || y0 > 4.0f * by + 3.0f) continue;
#pragma unroll
    for (int bx = 0; bx < 2; ++bx) {
      if (x1 < 8.0f * bx || x0 > 8.0f * bx + 7.0f) continue;
      if (!EXACT) {
        m |= 1u << (by * 2 + bx);
        continue;
      }
      const float q = conic_min_over_rect(a, b, c, 8.0f * bx - rx - 0.01f,
                                          8.0f * bx + 7.0f - rx + 0.01f,
                                          4.0f * by - ry - 0.01f, 4.0f * by + 3.0f - ry + 0.01f);
      if (q <= r2m) m |= 1u << (by * 2 + bx);
    }
  }
  return m;
}

__device__ __forceinline__ unsigned lanemask_lt_() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Compacts the batch positions whose mask has this warp's bit, in order.
// Lane l reads the masks of its P = B/32 consecutive positions P l .. P l +
// P - 1 as one 32-bit word (B = 128) or P/8 64-bit words (positions past the
// batch's count hold empty masks); an exclusive warp scan of the per-lane
// hit counts places each lane's hits in the list.
template <int B>
__device__ __forceinline__ int build_warp_list(const unsigned char* s_mask,
                                               typename ListEntry<B>::T* list) {
  static_assert(B == 128 || B == 256 || B == 512, "tile batch of 128, 256 or 512 splats");
  constexpr int P = B / 32;
  constexpr int NW = P >= 8 ? P / 8 : 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long bits[NW];
  int c = 0;
  if (P == 4) {
    const unsigned m = reinterpret_cast<const unsigned*>(s_mask)[lane];
    bits[0] = (m >> warp) & 0x01010101u;  // bit 8k: position 4l + k
    c = __popc((unsigned)bits[0]);
  } else {
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const unsigned long long m = reinterpret_cast<const unsigned long long*>(s_mask)[lane * NW + w];
      bits[w] = (m >> warp) & 0x0101010101010101ull;  // bit 8k: position P l + 8 w + k
      c += __popcll(bits[w]);
    }
  }
  int incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  int pos = incl - c;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    unsigned long long bw = bits[w];
    while (bw) {
      const int bb = __ffsll((long long)bw) - 1;
      list[pos++] = (typename ListEntry<B>::T)(P * lane + 8 * w + (bb >> 3));
      bw &= bw - 1;
    }
  }
  __syncwarp();
  return __shfl_sync(0xffffffffu, incl, 31);
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
  const int32_t* order;    // work-item order (global tile ids) or null
  const int32_t* view_tf;  // per-view table index (one image per view) or null
  const float4* lut;
  const float2* shade;     // per-record Blinn-Phong factors (s_d, s_s) or null
  int lut_size, n_tf;
  ViewMap vm;  // per-view tiles and output pixels (views may differ in size)
  float bg0, bg1, bg2;
};

// Loads tables [lut0, lut0 + ntg) into shared memory; slots past ntg and
// table indices outside [0, n_tf) read as fully transparent.
template <int TG>
__device__ __forceinline__ void stage_luts(const CompArgs& A, int lut0, int ntg, float4* s_lut) {
  const int L = A.lut_size;
  for (int e = threadIdx.x; e < TG * L; e += blockDim.x) {
    const int t = e / L, k = e - t * L, ti = lut0 + t;
    s_lut[e] = (t < ntg && ti >= 0 && ti < A.n_tf) ? __ldg(&A.lut[(int64_t)ti * L + k])
                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Stages splat `i` of the tile list into batch slot `s`: geometry,
// per-TF colour and A w (and, for the backward, the slopes), the exponent
// cutoff and the warp-block mask.  Returns the record index.
//
// The forward (BWD = false) reads the group's tables from shared memory
// (`lut`, TG tables of L entries, transparent where the group has no table).
// The backward reads them from global memory through the L1 cache (`lut`
// points at the group's first table; bit t of `valid` says whether table t
// exists, a missing one reads as transparent): the 16 KB this frees at four
// tables lets four backward CTAs share an SM instead of three.
//
// Shading (Eq. 2, LIT): the forward stages the shaded colour s_d C(v) + s_s;
// the backward stages the unshaded C(v) and (s_d, s_s) in s_sh, with the
// colour slopes already scaled by s_d.  Without shading s_sh is unused.
template <int TG, int B, bool BWD, bool LIT>
__device__ __forceinline__ uint32_t stage_splat(const CompArgs& A, int i, int s, const float4* lut,
                                                unsigned valid, float tx0, float ty0,
                                                float4* s_geo, float2* s_c, float4* s_col,
                                                float4* s_slope, float2* s_sh,
                                                unsigned char* s_mask) {
  const int L = A.lut_size;
  const uint32_t g = A.vals[i];
  const float4 ge = A.geo[g], au = A.aux[g];
  s_geo[s] = make_float4(ge.x, ge.y, -0.5f * au.x, -au.y);
  const TfPos q = tf_pos(au.w, L);
  const float sl = (au.w >= 0.0f && au.w <= 1.0f) ? (float)(L - 1) : 0.0f;
  float2 sh = make_float2(1.0f, 0.0f);
  if (LIT) sh = A.shade[g];
  if (LIT && BWD) s_sh[s] = sh;
  const float slc = LIT ? sl * sh.x : sl;  // colour slope scale
  float max_aw = 0.0f;
#pragma unroll
  for (int t = 0; t < TG; ++t) {
    float4 lo, hi;
    if (BWD) {
      const bool ok = (valid >> t) & 1u;
      lo = ok ? __ldg(&lut[t * L + q.k]) : make_float4(0.f, 0.f, 0.f, 0.f);
      hi = ok ? __ldg(&lut[t * L + q.k + 1]) : make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      lo = lut[t * L + q.k];
      hi = lut[t * L + q.k + 1];
    }
    const float Aop = lerp_rn(lo.w, hi.w, q);
    const float aw = mul(Aop, ge.w);
    float r = lerp_rn(lo.x, hi.x, q), gc = lerp_rn(lo.y, hi.y, q), b = lerp_rn(lo.z, hi.z, q);
    if (LIT && !BWD) {
      r = __fmaf_rn(sh.x, r, sh.y);
      gc = __fmaf_rn(sh.x, gc, sh.y);
      b = __fmaf_rn(sh.x, b, sh.y);
    }
    s_col[t * B + s] = make_float4(r, gc, b, aw);
    if (BWD)
      s_slope[t * B + s] = make_float4(slc * (hi.x - lo.x), slc * (hi.y - lo.y),
                                            slc * (hi.z - lo.z), ge.w * sl * (hi.w - lo.w));
    max_aw = fmaxf(max_aw, aw);
  }
  const float cut = power_cutoff(max_aw);
  s_c[s] = make_float2(-0.5f * au.z, cut);
  s_mask[s] = (unsigned char)warp_block_mask<BWD>(ge.x - tx0, ge.y - ty0, au.x, au.y, au.z, cut);
  return g;
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------

// stats (instrumented build): visited pairs (every pair reached before the
// pixel's termination, the method's own count), iterated pairs (walked by
// the warp lists), pairs above the cutoff, alpha evaluations, blended pairs.
//
// Resident CTAs per SM: 5 for one TF (48 registers; the extra CTA hides the
// batch barriers, 7% faster than 4 on the training step), 4 for 2-4 TFs,
// 2 for 8.
template <int TG, int B, bool STATS, bool LIT>
__global__ void __launch_bounds__(256, (TG >= 8 ? 2 : (TG == 1 ? 5 : 4)))
    composite_fwd_kernel(CompArgs A, float4* __restrict__ out,
                         int32_t* __restrict__ n_contrib, unsigned long long* __restrict__ stats) {
  pdl_enter();
  extern __shared__ float4 s_lut[];  // [TG][L]
  __shared__ float4 s_geo[B];        // u_x, u_y, -a/2, -b
  __shared__ float2 s_c[B];          // -c/2, exponent cutoff
  __shared__ float4 s_col[TG * B];
  __shared__ __align__(16) unsigned char s_mask[B];
  __shared__ typename ListEntry<B>::T s_list[kWarps][B];
  const int t0 = blockIdx.z * TG;  // first output image of the group
  const int ntg = A.view_tf ? 1 : min(TG, A.n_tf - t0);
  const int warp = threadIdx.x >> 5;
  unsigned long long n_vis = 0, n_it = 0, n_eval = 0, n_alpha = 0, n_blend = 0;
  {
    const int item = (int)blockIdx.x;
    const int wi = A.order ? A.order[item] : item;  // global tile id
    const int view = view_of_tile(A.vm, wi), tile = wi - A.vm.tile_off[view];
    const int tiles_x = A.vm.tiles_x[view], width = A.vm.width[view], height = A.vm.height[view];
    const long long pix0 = A.vm.pix_off[view];          // the view's first output pixel
    const int lut0 = A.view_tf ? A.view_tf[view] : t0;  // first table of the group
    stage_luts<TG>(A, lut0, ntg, s_lut);
    int px, py;
    pixel_of(tile, tiles_x, px, py);
    const float tx0 = (float)((tile % tiles_x) * VEG_TILE);
    const float ty0 = (float)((tile / tiles_x) * VEG_TILE);
    const bool inside = px < width && py < height;
    const float2 fxy = make_float2((float)px, (float)py);
    const int2 rg = A.ranges[wi];
    float T[TG], Cr[TG], Cg[TG], Cb[TG];
    int last[TG];
#pragma unroll
    for (int t = 0; t < TG; ++t) {
      T[t] = 1.0f;
      Cr[t] = Cg[t] = Cb[t] = 0.0f;
      last[t] = 0;
    }
    unsigned act = inside ? ((1u << ntg) - 1u) : 0u;

    for (int start = rg.x; start < rg.y; start += B) {
      if (__syncthreads_count(act != 0u) == 0) break;
      const int cnt = min(B, rg.y - start);
#pragma unroll
      for (int r = 0; r < (B + 255) / 256; ++r) {
        const int sl = (int)threadIdx.x + 256 * r;
        if (sl < cnt)
          stage_splat<TG, B, false, LIT>(A, start + sl, sl, s_lut, 0xffu, tx0, ty0, s_geo, s_c,
                                         s_col, nullptr, nullptr, s_mask);
        else if (sl < B)
          s_mask[sl] = 0;
      }
      __syncthreads();
      const int nw = build_warp_list<B>(s_mask, s_list[warp]);
      const bool act0 = act != 0u;
      int jstop = cnt;  // 1 + batch position where this pixel terminated
      // Eq. 1 update of every live TF of the group with splat j (exponent G).
      auto blend = [&](int j, float G) {
#pragma unroll
        for (int t = 0; t < TG; ++t) {
          if (!(act & (1u << t))) continue;
          if (STATS) ++n_alpha;
          const float4 c = s_col[t * B + j];
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
        if (STATS && !act) jstop = j + 1;
      };
      // four (then two, then one) splats per step: their exponents are
      // independent and overlap, the blends stay in list order
      int k = 0;
      for (; k + 3 < nw && act; k += 4) {
        const int j0 = s_list[warp][k], j1 = s_list[warp][k + 1];
        const int j2 = s_list[warp][k + 2], j3 = s_list[warp][k + 3];
        const float4 g0 = s_geo[j0], g1 = s_geo[j1], g2 = s_geo[j2], g3 = s_geo[j3];
        const float2 c0 = s_c[j0], c1 = s_c[j1], c2 = s_c[j2], c3 = s_c[j3];
        float2 d0, d1, d2, d3, q0, q1, q2, q3;
        float x0, x1, x2, x3;
        const float p0 = power_at(g0.x, g0.y, fxy, g0.z, g0.w, c0.x, d0, q0, x0);
        const float p1 = power_at(g1.x, g1.y, fxy, g1.z, g1.w, c1.x, d1, q1, x1);
        const float p2 = power_at(g2.x, g2.y, fxy, g2.z, g2.w, c2.x, d2, q2, x2);
        const float p3 = power_at(g3.x, g3.y, fxy, g3.z, g3.w, c3.x, d3, q3, x3);
        const bool e0 = !(p0 < c0.y || p0 > 0.0f), e1 = !(p1 < c1.y || p1 > 0.0f);
        const bool e2 = !(p2 < c2.y || p2 > 0.0f), e3 = !(p3 < c3.y || p3 > 0.0f);
        if (STATS) {
          n_it += 4;
          n_eval += (unsigned)e0 + (unsigned)e1 + (unsigned)e2 + (unsigned)e3;
        }
        if (e0) blend(j0, gauss_of(p0));
        if (e1 && act) blend(j1, gauss_of(p1));
        if (e2 && act) blend(j2, gauss_of(p2));
        if (e3 && act) blend(j3, gauss_of(p3));
      }
      for (; k + 1 < nw && act; k += 2) {
        const int j0 = s_list[warp][k], j1 = s_list[warp][k + 1];
        const float4 g0 = s_geo[j0], g1 = s_geo[j1];
        const float2 c0 = s_c[j0], c1 = s_c[j1];
        float2 d0, d1, q0, q1;
        float x0, x1;
        const float p0 = power_at(g0.x, g0.y, fxy, g0.z, g0.w, c0.x, d0, q0, x0);
        const float p1 = power_at(g1.x, g1.y, fxy, g1.z, g1.w, c1.x, d1, q1, x1);
        const bool e0 = !(p0 < c0.y || p0 > 0.0f), e1 = !(p1 < c1.y || p1 > 0.0f);
        if (STATS) {
          n_it += 2;
          n_eval += (unsigned)e0 + (unsigned)e1;
        }
        if (e0) blend(j0, gauss_of(p0));
        if (e1 && act) blend(j1, gauss_of(p1));
      }
      if (k < nw && act) {
        const int j = s_list[warp][k];
        const float4 sg = s_geo[j];
        const float2 sc = s_c[j];
        float2 d, d2;
        float dxy;
        const float power = power_at(sg.x, sg.y, fxy, sg.z, sg.w, sc.x, d, d2, dxy);
        if (STATS) ++n_it;
        if (!(power < sc.y || power > 0.0f)) {
          if (STATS) ++n_eval;
          blend(j, gauss_of(power));
        }
      }
      if (STATS && act0) n_vis += (unsigned long long)jstop;
    }
    if (inside) {
#pragma unroll
      for (int t = 0; t < TG; ++t) {
        if (t >= ntg) break;
        const int64_t o = pix0 + ((int64_t)(t0 + t) * height + py) * width + px;
        out[o] = make_float4(add(Cr[t], mul(T[t], A.bg0)), add(Cg[t], mul(T[t], A.bg1)),
                             add(Cb[t], mul(T[t], A.bg2)), T[t]);
        n_contrib[o] = last[t];
      }
    }
  }
  if (STATS) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n_vis += __shfl_down_sync(0xffffffffu, n_vis, o);
      n_it += __shfl_down_sync(0xffffffffu, n_it, o);
      n_eval += __shfl_down_sync(0xffffffffu, n_eval, o);
      n_alpha += __shfl_down_sync(0xffffffffu, n_alpha, o);
      n_blend += __shfl_down_sync(0xffffffffu, n_blend, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&stats[0], n_vis);
      atomicAdd(&stats[1], n_it);
      atomicAdd(&stats[2], n_eval);
      atomicAdd(&stats[3], n_alpha);
      atomicAdd(&stats[4], n_blend);
    }
  }
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------

// Sums eight per-lane values over the warp with 9 shuffles: three halving
// exchanges (offsets 16, 8, 4; each lane keeps the half named by its offset
// bit and receives the partner's sum of that half), then two full steps
// (offsets 2, 1).  Lane l returns the warp total of slot l >> 2.
__device__ __forceinline__ float warp_reduce_scatter8(const float v[8], int lane) {
  const bool b4 = lane & 16, b2 = lane & 8, b1 = lane & 4;
  float w[4], x[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = b4 ? v[i] : v[i + 4];
    const float keep = b4 ? v[i + 4] : v[i];
    w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = b2 ? w[i] : w[i + 2];
    const float keep = b2 ? w[i + 2] : w[i];
    x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const float send = b1 ? x[0] : x[1];
  float y = (b1 ? x[1] : x[0]) + __shfl_xor_sync(0xffffffffu, send, 4);
  y += __shfl_xor_sync(0xffffffffu, y, 2);
  y += __shfl_xor_sync(0xffffffffu, y, 1);
  return y;
}

// The same for sixteen values with 16 shuffles (halving at offsets 16, 8, 4,
// 2, then one full step at offset 1).  Lane l returns the warp total of
// slot l >> 1.
__device__ __forceinline__ float warp_reduce_scatter16(const float v[16], int lane) {
  const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4, b2 = lane & 2;
  float w[8], x[4], y[2];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float send = b16 ? v[i] : v[i + 8];
    const float keep = b16 ? v[i + 8] : v[i];
    w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = b8 ? w[i] : w[i + 4];
    const float keep = b8 ? w[i + 4] : w[i];
    x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = b4 ? x[i] : x[i + 2];
    const float keep = b4 ? x[i + 2] : x[i];
    y[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  const float send = b2 ? y[0] : y[1];
  float z = (b2 ? y[1] : y[0]) + __shfl_xor_sync(0xffffffffu, send, 2);
  z += __shfl_xor_sync(0xffffffffu, z, 1);
  return z;
}

// Sums one value per splat for two splats (a, b) over the warp with 5
// shuffles (one halving exchange at offset 16, then full steps at 8, 4, 2,
// 1).  Lanes 0-15 return the total of a, lanes 16-31 that of b.
__device__ __forceinline__ float warp_reduce_pair(float a, float b, int lane) {
  const bool hi = lane & 16;
  float x = (hi ? b : a) + __shfl_xor_sync(0xffffffffu, hi ? a : b, 16);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ void red_add_v2(float2* p, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

__device__ __forceinline__ void red_add_v4(float4* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
               "f"(d)
               : "memory");
}

// Walks each pixel's list back to front, from its last contribution to the
// first splat.  Below n_contrib a pair blends exactly when its exponent is in
// range and alpha >= 1/255 (the stop only ends the list), so every decision
// is recomputed bit for bit from the same float32 operations as the forward,
// without the forward's transmittance.  With T_i the transmittance in front
// of blended splat i and Suf_i = sum over blended j > i of (c_j . g) alpha_j
// T_j + T_final (bg . g + g_T), the gradient of the loss w.r.t. alpha_i is
//   dL/dalpha_i = T_i (c_i . g) - Suf_i / (1 - alpha_i).
// Each pixel starts from T_final (the forward's output) and recovers
// T_i = T_{i+1} / (1 - alpha_i) with the reciprocal that dL/dalpha_i needs
// anyway; Suf grows from the back, so the small terms of deep splats are
// summed first and keep their relative accuracy (a front-to-back prefix
// K - S_i would leave them as a difference of two O(1) numbers).  Per splat,
// the seven screen-space gradients are reduced over the warp, summed over
// warps in shared memory and added to the per-record gradient buffer once
// per tile.
//
// The weight needs no sum of its own: below the clamp alpha = A w e^power,
// so dalpha/dw = alpha / w = (dalpha/dpower) / w and dL/dw is the summed
// exponent gradient dL/dpower divided by w (applied at the flush; a splat
// with w = 0 never blends and gets 0).
//
// Shaded (LIT): the blended colour is s_d C + s_s, so c.g = s_d (C.g) + s_s
// (g_r + g_g + g_b), dL/dC = s_d alpha T g, and the pair adds alpha T (C.g)
// to dL/ds_d and alpha T (g_r + g_g + g_b) to dL/ds_s.  dL/ds_d takes the
// eighth slot of the 16-slot reduce-scatter and dL/ds_s a separate pair
// reduction; the two shading sums go to grad_shade.
//
// stats (instrumented build): replayed pairs (list positions below the
// pixel's last contribution), iterated pairs, pairs above the cutoff, alpha
// evaluations, blended pairs, blended pairs below the clamp, pairs with a
// nonzero screen-space gradient.
//
// Resident CTAs per SM: 4 (64 registers; 8 warps per SM more than 3 CTAs
// hide the walk's dependent-issue latency, 7% faster on the training step),
// 3 for the shaded and instrumented builds of a 4-TF group, which would
// spill at 64 registers.
template <int TG, int B, bool STATS, bool LIT>
__global__ void __launch_bounds__(256, ((LIT || STATS) && TG >= 4) ? 3 : 4)
    composite_bwd_kernel(CompArgs A, const float4* __restrict__ out,
                         const int32_t* __restrict__ n_contrib, const float4* __restrict__ dout,
                         float4* __restrict__ grad2d, float2* __restrict__ grad_shade,
                         unsigned long long* __restrict__ stats) {
  pdl_enter();
  constexpr int kAcc = LIT ? 12 : 8;  // accumulator slots per splat
  unsigned long long n_rep = 0, n_it = 0, n_eval = 0, n_alpha = 0, n_blend = 0, n_free = 0,
                     n_grad = 0;
  extern __shared__ float4 smem[];
  using LT = typename ListEntry<B>::T;
  float4* s_col = smem;                                // [TG][B]: rgb, A w
  float4* s_slope = s_col + TG * B;                    // [TG][B]: drgb/dv, w dA/dv
  float4* s_geo = s_slope + TG * B;                    // [B]: u, -a/2, -b
  float2* s_c = reinterpret_cast<float2*>(s_geo + B);  // [B]: -c/2, cutoff
  float2* s_sh = s_c + B;                              // [B]: s_d, s_s (LIT)
  float* s_acc = reinterpret_cast<float*>(s_sh + (LIT ? B : 0));  // [B][kAcc] gradient sums
  uint32_t* s_idx = reinterpret_cast<uint32_t*>(s_acc + kAcc * B);  // [B]: record index
  unsigned char* s_mask = reinterpret_cast<unsigned char*>(s_idx + B);  // [B]
  LT* s_lists = reinterpret_cast<LT*>(s_mask + B);  // [kWarps][B]
  __shared__ int s_maxnc;

  const int t0 = blockIdx.z * TG;  // first output image of the group
  const int ntg = A.view_tf ? 1 : min(TG, A.n_tf - t0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  LT* my_list = s_lists + warp * B;
  for (int e = threadIdx.x; e < kAcc * B; e += 256) s_acc[e] = 0.0f;
  {
    const int item = (int)blockIdx.x;
    const int wi = A.order ? A.order[item] : item;  // global tile id
    const int view = view_of_tile(A.vm, wi), tile = wi - A.vm.tile_off[view];
    const int tiles_x = A.vm.tiles_x[view], width = A.vm.width[view], height = A.vm.height[view];
    const long long pix0 = A.vm.pix_off[view];          // the view's first output pixel
    const int lut0 = A.view_tf ? A.view_tf[view] : t0;  // first table of the group
    const float4* g_lut = A.lut + (int64_t)lut0 * A.lut_size;  // the group's tables
    unsigned valid = 0u;
#pragma unroll
    for (int t = 0; t < TG; ++t)
      if (t < ntg && lut0 + t >= 0 && lut0 + t < A.n_tf) valid |= 1u << t;
    if (threadIdx.x == 0) s_maxnc = 0;
    int px, py;
    pixel_of(tile, tiles_x, px, py);
    const float tx0 = (float)((tile % tiles_x) * VEG_TILE);
    const float ty0 = (float)((tile / tiles_x) * VEG_TILE);
    const bool inside = px < width && py < height;
    const float2 fxy = make_float2((float)px, (float)py);
    const int2 rg = A.ranges[wi];

    // per TF: transmittance behind the splats walked so far, the suffix sum,
    // the upstream colour gradient and n_contrib
    float T[TG], Suf[TG], gr[TG], gg[TG], gb[TG], gs[TG];
    int nc[TG];
    int my_max = 0;
#pragma unroll
    for (int t = 0; t < TG; ++t) {
      T[t] = 1.0f;
      Suf[t] = 0.0f;
      gr[t] = gg[t] = gb[t] = gs[t] = 0.0f;
      nc[t] = 0;
      if (inside && t < ntg) {
        const int64_t o = pix0 + ((int64_t)(t0 + t) * height + py) * width + px;
        const float4 ov = out[o], dv4 = dout[o];
        nc[t] = n_contrib[o];
        gr[t] = dv4.x;
        gg[t] = dv4.y;
        gb[t] = dv4.z;
        gs[t] = dv4.x + dv4.y + dv4.z;
        T[t] = ov.w;
        Suf[t] = ov.w * (A.bg0 * dv4.x + A.bg1 * dv4.y + A.bg2 * dv4.z + dv4.w);
        my_max = max(my_max, nc[t]);
      }
    }
    if (STATS) n_rep += (unsigned long long)my_max;
    // loop bounds: a warp walks from its last contribution (all lanes take part
    // in the reductions); the block stages from its last warp's
    int warp_max = my_max;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      warp_max = max(warp_max, __shfl_xor_sync(0xffffffffu, warp_max, o));
    __syncthreads();
    if (lane == 0) atomicMax(&s_maxnc, warp_max);
    __syncthreads();
    const int block_max = s_maxnc;

    // batches from the back: list positions [bstart, bend), slot s = bstart + s
    for (int bend = block_max; bend > 0; bend -= B) {
      const int bstart = max(0, bend - B);
      const int cnt = bend - bstart;
#pragma unroll
      for (int r = 0; r < (B + 255) / 256; ++r) {
        const int sl = (int)threadIdx.x + 256 * r;
        if (sl < cnt)
          s_idx[sl] = stage_splat<TG, B, true, LIT>(A, rg.x + bstart + sl, sl, g_lut, valid, tx0,
                                                    ty0, s_geo, s_c, s_col, s_slope, s_sh, s_mask);
        else if (sl < B)
          s_mask[sl] = 0;
      }
      __syncthreads();
      const int nw = build_warp_list<B>(s_mask, my_list);
      // blend of splat j at list position idx, undone for every TF of the
      // group: accumulates dL/dG, dL/dv (and dL/ds_d, dL/ds_s) of this pixel
      auto tf_grads = [&](int j, int idx, float G, float& dG, float& dvv, float& dsd,
                          float& dss) {
        float2 sh = make_float2(1.0f, 0.0f);
        if (LIT) sh = s_sh[j];
#pragma unroll
        for (int t = 0; t < TG; ++t) {
          if (idx >= nc[t]) continue;
          if (STATS) ++n_alpha;
          const float4 c = s_col[t * B + j];
          const float raw = mul(c.w, G);
          const float alpha = fminf(kAlphaMax, raw);
          if (alpha < kAlphaMin) continue;
          if (STATS) {
            ++n_blend;
            n_free += (raw <= kAlphaMax);
          }
          const float rr = rcp_approx(sub(1.0f, alpha));
          const float Ti = T[t] * rr;  // transmittance in front of the splat
          const float wgt = alpha * Ti;
          const float cgu = c.x * gr[t] + c.y * gg[t] + c.z * gb[t];
          const float cgd = LIT ? sh.x * cgu + sh.y * gs[t] : cgu;
          if (LIT) {
            dsd += wgt * cgu;
            dss += wgt * gs[t];
          }
          const float dalpha = Ti * cgd - Suf[t] * rr;
          Suf[t] = __fmaf_rn(cgd, wgt, Suf[t]);
          const float4 sl = s_slope[t * B + j];
          dvv += wgt * (gr[t] * sl.x + gg[t] * sl.y + gb[t] * sl.z);
          if (raw <= kAlphaMax) {
            dvv += dalpha * G * sl.w;
            dG += dalpha * c.w;
          }
          T[t] = Ti;
        }
      };
      // gradient parts of one pair: the exponent gradient dp = dL/dpower
      // times the offset moments dx, dy, dx^2, dx dy, dy^2 (d = u - pixel),
      // dL/dv, dp itself (dL/dw times w) (and s_d).  The screen gradients
      // are linear in these moments with per-splat coefficients (power =
      // -a/2 dx^2 - b dx dy - c/2 dy^2), applied once per splat at the flush.
      auto pair_parts = [&](float* v, float dp, float2 d, float2 d2, float dxy, float dvv,
                            float dsd) {
        const float2 m = mul2(make_float2(dp, dp), d);
        v[0] = m.x;
        v[1] = m.y;
        v[2] = dp * d2.x;
        v[3] = dp * dxy;
        v[4] = dp * d2.y;
        v[5] = dvv;
        v[6] = dp;
        v[7] = LIT ? dsd : 0.0f;
      };
      // the warp's list is in list order: skip its entries past the warp's
      // last contribution, then walk it backwards two splats per step (j0, the
      // later one, first); independent geometry and exponentials overlap, and
      // one 16-slot reduce-scatter sums both splats' gradients over the warp
      int k = nw - 1;
      while (k >= 0 && bstart + my_list[k] >= warp_max) --k;
      for (; k >= 0; k -= 2) {
        const int j0 = my_list[k];
        const int idx0 = bstart + j0;  // list position
        const bool has1 = k >= 1;
        const int j1 = has1 ? my_list[k - 1] : j0;
        const int idx1 = bstart + j1;
        if (STATS) n_it += 1 + (unsigned)has1;
        const float4 sg0 = s_geo[j0], sg1 = s_geo[j1];
        const float2 sc0 = s_c[j0], sc1 = s_c[j1];
        float2 d0, d1, q0, q1;
        float x0, x1;
        const float p0 = power_at(sg0.x, sg0.y, fxy, sg0.z, sg0.w, sc0.x, d0, q0, x0);
        const float p1 = power_at(sg1.x, sg1.y, fxy, sg1.z, sg1.w, sc1.x, d1, q1, x1);
        const bool ev0 = idx0 < my_max && p0 <= 0.0f && p0 >= sc0.y;
        const bool ev1 = has1 && idx1 < my_max && p1 <= 0.0f && p1 >= sc1.y;
        const float G0 = ev0 ? gauss_of(p0) : 0.f;
        const float G1 = ev1 ? gauss_of(p1) : 0.f;
        float dG0 = 0.f, dv0 = 0.f, dG1 = 0.f, dv1 = 0.f;
        float dd0 = 0.f, ds0 = 0.f, dd1 = 0.f, ds1 = 0.f;
        if (ev0) tf_grads(j0, idx0, G0, dG0, dv0, dd0, ds0);
        if (ev1) tf_grads(j1, idx1, G1, dG1, dv1, dd1, ds1);
        if (STATS) n_eval += (unsigned)ev0 + (unsigned)ev1;
        if (STATS) n_grad += (unsigned)(dG0 != 0.f) + (unsigned)(dG1 != 0.f);
        const float dp0 = dG0 * G0, dp1 = dG1 * G1;
        bool nz = dp0 != 0.f || dv0 != 0.f || dp1 != 0.f || dv1 != 0.f;
        if (LIT) nz = nz || dd0 != 0.f || ds0 != 0.f || dd1 != 0.f || ds1 != 0.f;
        if (__any_sync(0xffffffffu, nz)) {
          float v[16];
          pair_parts(v, dp0, d0, q0, x0, dv0, dd0);
          pair_parts(v + 8, dp1, d1, q1, x1, dv1, dd1);
          // lane l ends with slot l >> 1 (splat (l >> 4), component (l >> 1) & 7)
          const float r = warp_reduce_scatter16(v, lane);
          const int slot = lane >> 1, which = slot >> 3, comp = slot & 7;
          if ((lane & 1) == 0 && comp < (LIT ? 8 : 7) && (which == 0 || has1))
            atomicAdd(&s_acc[(which ? j1 : j0) * kAcc + comp], r);
          if (LIT) {
            const float rs = warp_reduce_pair(ds0, ds1, lane);
            if ((lane & 15) == 1 && (lane < 16 || has1))
              atomicAdd(&s_acc[(lane < 16 ? j0 : j1) * kAcc + 8], rs);
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < (B + 255) / 256; ++r) {
        const int sl = (int)threadIdx.x + 256 * r;
        if (sl >= cnt) break;
        float4* acc = reinterpret_cast<float4*>(s_acc) + (kAcc / 4) * sl;
        const float4 a0 = acc[0], a1 = acc[1];
        const float4 a2 = LIT ? acc[2] : make_float4(0.f, 0.f, 0.f, 0.f);
        acc[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        acc[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (LIT) acc[2] = make_float4(0.f, 0.f, 0.f, 0.f);
        const bool any = a0.x != 0.f || a0.y != 0.f || a0.z != 0.f || a0.w != 0.f ||
                         a1.x != 0.f || a1.y != 0.f || a1.z != 0.f;
        const uint32_t rec = s_idx[sl];
        if (any) {
          // moments (S_x, S_y, S_xx, S_xy, S_yy) of dp to the screen
          // gradients: du = (-a S_x - b S_y, -b S_x - c S_y), dconic =
          // (-S_xx / 2, -S_xy, -S_yy / 2); s_geo holds (u, -a/2, -b), s_c -c/2
          const float4 sg = s_geo[sl];
          const float sc = s_c[sl].x;
          float4* dst = grad2d + 2 * (int64_t)rec;
          const float w = A.geo[rec].w;
          const float dw = w > 0.0f ? a1.z / w : 0.0f;
          red_add_v4(dst, 2.0f * sg.z * a0.x + sg.w * a0.y, 2.0f * sc * a0.y + sg.w * a0.x,
                     -0.5f * a0.z, -a0.w);
          red_add_v4(dst + 1, -0.5f * a1.x, a1.y, dw, 0.0f);
        }
        if (LIT && (a1.w != 0.f || a2.x != 0.f)) red_add_v2(grad_shade + rec, a1.w, a2.x);
      }
      __syncthreads();
    }
  }
  if (STATS) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n_rep += __shfl_down_sync(0xffffffffu, n_rep, o);
      n_it += __shfl_down_sync(0xffffffffu, n_it, o);
      n_eval += __shfl_down_sync(0xffffffffu, n_eval, o);
      n_alpha += __shfl_down_sync(0xffffffffu, n_alpha, o);
      n_blend += __shfl_down_sync(0xffffffffu, n_blend, o);
      n_free += __shfl_down_sync(0xffffffffu, n_free, o);
      n_grad += __shfl_down_sync(0xffffffffu, n_grad, o);
    }
    if (lane == 0) {
      atomicAdd(&stats[0], n_rep);
      atomicAdd(&stats[1], n_it);
      atomicAdd(&stats[2], n_eval);
      atomicAdd(&stats[3], n_alpha);
      atomicAdd(&stats[4], n_blend);
      atomicAdd(&stats[5], n_free);
      atomicAdd(&stats[6], n_grad);
    }
  }
}

size_t bwd_smem_bytes(int TG, int L, bool lit, int B) {
  // col + slope, geo, (c, cutoff), (s_d, s_s), acc, idx, mask, warp lists (the
  // tables stay in global memory)
  (void)L;
  return (size_t)TG * B * 16 * 2 + (size_t)B * 16 + (size_t)B * 8 +
         (lit ? (size_t)B * 8 : 0) + (size_t)(lit ? 12 : 8) * B * 4 + (size_t)B * 4 +
         (size_t)B + (size_t)kWarps * B * (B > 256 ? 2 : 1);
}

// Shared memory of a forward CTA: the group's tables (dynamic) and the
// batch arrays (static).
size_t fwd_smem_bytes(int TG, int L, int B) {
  return (size_t)TG * L * 16 + (size_t)B * (16 + 8 + 1) + (size_t)TG * B * 16 +
         (size_t)kWarps * B * (B > 256 ? 2 : 1);
}

// Tile batch: the caller's choice (128, 256 or 512 splats), else 256.
int pick_batch(int tile_batch) { return tile_batch == 128 || tile_batch == 512 ? tile_batch : 256; }

// TF group size: the caller's choice, else 1 for the forward (measured
// fastest at the training-step and sweep shapes: each TF stops at its own
// termination) and up to 4 for the backward (whose replay shares each
// splat's geometry and reductions across the group); halved until the
// group's shared memory fits one CTA (227 KB) at tile batch B.  The group
// size changes no result; one table of up to 4096 entries always fits.
int pick_group(int tf_group, int n_tf, bool bwd, int lut_size, bool lit, int B) {
  int g = tf_group;
  if (g <= 0) g = bwd ? std::min(n_tf, 4) : 1;
  g = g <= 1 ? 1 : g <= 2 ? 2 : (g <= 4 || bwd) ? 4 : 8;
  auto fits = [&](int tg) {
    const size_t bytes = bwd ? bwd_smem_bytes(tg, lut_size, lit, B) + 1024
                             : fwd_smem_bytes(tg, lut_size, B) + 1024;
    return bytes <= (size_t)227 * 1024;
  };
  while (g > 1 && !fits(g)) g /= 2;
  return g;
}

CompArgs make_args(const veg_camera* cams, int n_views, const float4* geo, const float4* aux,
                   const uint32_t* vals, const int2* ranges, const int32_t* order, veg_tf tf,
                   const float* bg, const float* shade) {
  CompArgs A;
  A.shade = reinterpret_cast<const float2*>(shade);
  A.geo = geo;
  A.aux = aux;
  A.vals = vals;
  A.ranges = ranges;
  A.order = order;
  A.view_tf = tf.view_tf;
  A.lut = reinterpret_cast<const float4*>(tf.lut);
  A.lut_size = tf.lut_size;
  A.n_tf = tf.n_tf;
  A.vm = make_viewmap(cams, n_views, tf.view_tf ? 1 : tf.n_tf);
  A.bg0 = bg ? bg[0] : 0.f;
  A.bg1 = bg ? bg[1] : 0.f;
  A.bg2 = bg ? bg[2] : 0.f;
  return A;
}

template <int TG, int B, bool STATS, bool LIT>
veg_status launch_fwd_t(const CompArgs& A, int n_views, float4* out, int32_t* nc,
                        unsigned long long* stats, cudaStream_t stream) {
  const size_t smem = (size_t)TG * A.lut_size * sizeof(float4);
  auto kern = composite_fwd_kernel<TG, B, STATS, LIT>;
  static SmemRecord configured;
  veg_status st = prepare_smem(kern, smem, configured, true);
  if (st != VEG_OK) return st;
  const unsigned groups = A.view_tf ? 1u : (unsigned)((A.n_tf + TG - 1) / TG);
  dim3 grid((unsigned)A.vm.tile_off[n_views], 1u, groups);
  launch_k(kern, grid, 256, smem, stream, A, out, nc, stats);
  count_launch();
  return launch_status();
}

template <int TG, int B, bool STATS, bool LIT>
veg_status launch_bwd_t(const CompArgs& A, int n_views, const float4* out, const int32_t* nc,
                        const float4* dout, float4* grad2d, float2* grad_shade,
                        unsigned long long* stats, cudaStream_t stream) {
  const size_t smem = bwd_smem_bytes(TG, A.lut_size, LIT, B);
  auto kern = composite_bwd_kernel<TG, B, STATS, LIT>;
  static SmemRecord configured;
  veg_status st = prepare_smem(kern, smem, configured, true);
  if (st != VEG_OK) return st;
  const unsigned groups = A.view_tf ? 1u : (unsigned)((A.n_tf + TG - 1) / TG);
  dim3 grid((unsigned)A.vm.tile_off[n_views], 1u, groups);
  launch_k(kern, grid, 256, smem, stream, A, out, nc, dout, grad2d, grad_shade, stats);
  count_launch();
  return launch_status();
}

// Dispatch over the tile batch (the instrumented builds use 256: the pair
// counts do not depend on the batch).
template <int TG, bool STATS, bool LIT>
veg_status fwd_batch(int B, const CompArgs& A, int n_views, float4* out, int32_t* nc,
                     unsigned long long* stats, cudaStream_t stream) {
  if constexpr (!STATS) {
    if (B == 128) return launch_fwd_t<TG, 128, STATS, LIT>(A, n_views, out, nc, stats, stream);
    if (B == 512) return launch_fwd_t<TG, 512, STATS, LIT>(A, n_views, out, nc, stats, stream);
  }
  return launch_fwd_t<TG, 256, STATS, LIT>(A, n_views, out, nc, stats, stream);
}

template <int TG, bool STATS, bool LIT>
veg_status bwd_batch(int B, const CompArgs& A, int n_views, const float4* out, const int32_t* nc,
                     const float4* dout, float4* grad2d, float2* grad_shade,
                     unsigned long long* stats, cudaStream_t stream) {
  if constexpr (!STATS) {
    if (B == 128)
      return launch_bwd_t<TG, 128, STATS, LIT>(A, n_views, out, nc, dout, grad2d, grad_shade,
                                               stats, stream);
    if (B == 512)
      return launch_bwd_t<TG, 512, STATS, LIT>(A, n_views, out, nc, dout, grad2d, grad_shade,
                                               stats, stream);
  }
  return launch_bwd_t<TG, 256, STATS, LIT>(A, n_views, out, nc, dout, grad2d, grad_shade, stats,
                                           stream);
}

}  // namespace

}  // namespace veg
