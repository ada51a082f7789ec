// Shared internals of the VEG CUDA library: host-side launch bookkeeping,
// workspace carving, and the device-side float32 helpers whose operation
// order defines the binning-critical arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "veg.h"

namespace veg {

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

void count_launch(int k = 1);

// Returns VEG_ERR_CUDA if the last launch failed to enqueue.
veg_status launch_status();

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Largest dynamic shared-memory size one kernel has been configured for, per
// device (the attribute belongs to the function on each device).  The slow
// path holds a lock, so the attribute only grows under concurrent callers.
struct SmemRecord {
  static constexpr int kDevices = 64;
  std::atomic<size_t> bytes[kDevices];
  std::mutex lock;
};

// Allows `dyn` bytes of dynamic shared memory for `kern` on the current
// device (and, with max_carveout, prefers the largest shared-memory
// carveout), once per size increase; refuses sizes beyond the 227 KB a CTA
// may hold.
template <typename K>
veg_status prepare_smem(K kern, size_t dyn, SmemRecord& rec, bool max_carveout) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= SmemRecord::kDevices)
    return VEG_ERR_CUDA;
  if (dyn <= rec.bytes[dev].load(std::memory_order_acquire)) return VEG_OK;
  std::lock_guard<std::mutex> guard(rec.lock);
  if (dyn <= rec.bytes[dev].load(std::memory_order_acquire)) return VEG_OK;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return VEG_ERR_CUDA;
  if (fa.sharedSizeBytes + dyn > 227 * 1024) return VEG_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) !=
      cudaSuccess)
    return VEG_ERR_UNSUPPORTED;
  if (max_carveout && cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                           (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    return VEG_ERR_UNSUPPORTED;
  rec.bytes[dev].store(dyn, std::memory_order_release);
  return VEG_OK;
}

// Programmatic dependent launch.  Every kernel of the library starts with
// pdl_enter(): it waits until the kernel before it in the stream has
// finished and its writes are visible, then lets the next kernel be
// scheduled early (both are no-ops for a kernel launched without the
// attribute).  launch_k launches with the attribute, so a kernel's launch
// and block scheduling overlap the tail of the one before it.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... P, typename... A>
void launch_k(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
              A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, static_cast<A&&>(args)...);
}

// Bump allocator over a caller-provided workspace (256-byte aligned pieces).
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = round_up(off, 256);
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += count * sizeof(T);
    return p;
  }
  size_t bytes() const { return round_up(off, 256); }
};

// Status header at the start of a bin_sort / render workspace.
struct WsHeader {
  unsigned long long n_instances;  // total tile instances of the last binning
  unsigned int flags;              // VEG_FLAG_* bits
  unsigned int pad0;
  unsigned long long n_visible;    // records that touch a tile (last binning)
  unsigned int key_min, key_max;   // range of the depth sort's keys (last binning)
  unsigned int pad[56];
};
static_assert(sizeof(WsHeader) == 256, "header must be 256 bytes");
constexpr unsigned int FLAG_CAPACITY = 1u;
constexpr unsigned int FLAG_TIMEOUT = 2u;  // a bounded device-side wait gave up

struct CamParam {
  float r[9];
  float t[3];
  float fx, fy, cx, cy;
  float near_plane;
  int width, height, tiles_x, tiles_y;
};

struct CamSet {
  CamParam c[VEG_MAX_VIEWS];
};

// Views of one call may differ in image size.  Their tiles are numbered
// one view after another: view v owns the global tile ids [tile_off[v],
// tile_off[v + 1]), row-major in its own tile grid, and its n_out images of
// height[v] x width[v] pixels start at pixel pix_off[v] of the output.  For
// views of one size this is the layout [V][tiles] and [V][T][H][W].
struct ViewMap {
  int n_views;
  int tile_off[VEG_MAX_VIEWS + 1];
  int tiles_x[VEG_MAX_VIEWS];
  int width[VEG_MAX_VIEWS];
  int height[VEG_MAX_VIEWS];
  long long pix_off[VEG_MAX_VIEWS + 1];
  int max_tiles;  // the largest view's tile count
};

veg_status check_cameras(const veg_camera* cams, int32_t n_views);
// check_cameras, and every view of the size of the first
veg_status check_cameras_one_size(const veg_camera* cams, int32_t n_views);
void fill_camset(const veg_camera* cams, int32_t n_views, CamSet* out);

inline int tiles_x_of(int w) { return (w + VEG_TILE - 1) / VEG_TILE; }
inline int tile_bits_of(int tiles) {
  int b = 1;
  while ((1 << b) < tiles) ++b;
  return b;
}

// Tile total of the views (int64: callers check it against 2^31).
inline int64_t total_tiles_of(const veg_camera* cams, int n_views) {
  int64_t t = 0;
  for (int v = 0; v < n_views; ++v)
    t += (int64_t)tiles_x_of(cams[v].width) * tiles_x_of(cams[v].height);
  return t;
}

// images_per_view: output images of each view (the TFs of the call, or one).
inline ViewMap make_viewmap(const veg_camera* cams, int n_views, int images_per_view) {
  ViewMap m;
  m.n_views = n_views;
  m.tile_off[0] = 0;
  m.pix_off[0] = 0;
  m.max_tiles = 0;
  for (int v = 0; v < n_views; ++v) {
    const int tx = tiles_x_of(cams[v].width), t = tx * tiles_x_of(cams[v].height);
    m.tiles_x[v] = tx;
    m.width[v] = cams[v].width;
    m.height[v] = cams[v].height;
    m.tile_off[v + 1] = m.tile_off[v] + t;
    m.pix_off[v + 1] = m.pix_off[v] + (long long)images_per_view * cams[v].width *
                                          cams[v].height;
    m.max_tiles = t > m.max_tiles ? t : m.max_tiles;
  }
  return m;
}

// The view owning global tile id g (binary search over the view offsets).
__device__ __forceinline__ int view_of_tile(const ViewMap& m, int g) {
  int lo = 0, hi = m.n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (m.tile_off[mid] <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Entry points shared between translation units (no argument validation).
// Per-view models of one projection call (views may show different models).
struct ViewModels {
  const float4* mean_v[VEG_MAX_VIEWS];
  const float4* logscale_w[VEG_MAX_VIEWS];
  const float4* quat[VEG_MAX_VIEWS];
  int64_t n[VEG_MAX_VIEWS];
};

veg_status project_launch(const CamSet& cs, int n_views, veg_gaussians g, const veg_tf* cull_tf,
                          float4* geo, float4* aux, int32_t* tiles, short4* rect,
                          cudaStream_t stream);
size_t binsort_ws_bytes(int64_t n, int n_views, int64_t capacity);
veg_status binsort_launch(const veg_camera* cams, int n_views, int64_t n, const float4* geo,
                          const int32_t* tiles, const short4* rect, void* ws, int64_t capacity,
                          uint64_t* keys, uint32_t* vals, int2* ranges, cudaStream_t stream);
veg_status composite_fwd_launch(const veg_camera* cams, int n_views, int64_t n,
                                const float4* geo, const float4* aux, const uint32_t* vals,
                                const int2* ranges, const int32_t* order, veg_tf tf,
                                const float* bg, const float* shade, int tf_group,
                                int tile_batch, float4* out, int32_t* n_contrib,
                                unsigned long long* stats, cudaStream_t stream);
veg_status tile_order_launch(const int2* ranges, int count, int32_t* order, cudaStream_t stream);

// ---------------------------------------------------------------------------
// device side: float32 operations in a fixed order (no contraction)
// ---------------------------------------------------------------------------

__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float dv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }

// Paired float32 operations (one f32x2 instruction on sm_100-family GPUs);
// each half is rounded exactly like its scalar counterpart above.
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 d;
  asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
// a * b + c with one rounding per half
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

__device__ __forceinline__ float dot3(float a0, float a1, float a2, float b0, float b1,
                                      float b2) {
  return add(add(mul(a0, b0), mul(a1, b1)), mul(a2, b2));
}

// exp(x) by Cody-Waite reduction with ln 2 split into a 15-bit high part
// (exact products n * hi for |n| <= 256) and the remainder, then a degree-7
// Taylor polynomial in Horner form; scaling by 2^n through the exponent
// field.  Input clamped to [-80, 80].  Error <= 2 ulp (checked on the host
// against a float64 reference by the test suite).
__device__ __forceinline__ float exp_cw(float x) {
  const float kLog2e = 1.44269502162933349609375f;  // float32(log2 e)
  const float kLn2Hi = 0.693145751953125f;
  const float kLn2Lo = 1.428606765330187045037746429443359375e-06f;  // float32(ln2 - hi)
  x = fminf(fmaxf(x, -80.0f), 80.0f);
  float n = rintf(mul(x, kLog2e));
  float r = sub(x, mul(n, kLn2Hi));
  r = sub(r, mul(n, kLn2Lo));
  float p = 1.0f / 5040.0f;
  p = add(mul(p, r), 1.0f / 720.0f);
  p = add(mul(p, r), 1.0f / 120.0f);
  p = add(mul(p, r), 1.0f / 24.0f);
  p = add(mul(p, r), 1.0f / 6.0f);
  p = add(mul(p, r), 0.5f);
  p = add(mul(p, r), 1.0f);
  p = add(mul(p, r), 1.0f);
  int ni = (int)n;
  float scale = __int_as_float((ni + 127) << 23);
  return mul(p, scale);
}

// Linear interpolation of one RGBA table at v in float32 (fixed order).
// Entries sit at v = k/(L-1); v is clamped to [0, 1].
struct TfPos {
  int k;
  float tau, one_m;
};
__device__ __forceinline__ TfPos tf_pos(float v, int L) {
  float vc = fminf(fmaxf(v, 0.0f), 1.0f);
  float p = mul(vc, (float)(L - 1));
  float kf = fminf(floorf(p), (float)(L - 2));
  TfPos r;
  r.k = (int)kf;
  r.tau = sub(p, kf);
  r.one_m = sub(1.0f, r.tau);
  return r;
}
__device__ __forceinline__ float lerp_rn(float lo, float hi, const TfPos& q) {
  return add(mul(q.one_m, lo), mul(q.tau, hi));
}

constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kDilation = 0.3f;
constexpr float kFrustumSlack = 1.3f;
constexpr float kLambdaFloor = 0.1f;

}  // namespace veg
