// Tile binning and depth ordering for the tile rasteriser (Sec. 3.3).
//
// The required order is the stable sort of one 64-bit key per
// (Gaussian, tile) pair, key = (view, tile, depth bits), emitted in Gaussian
// index order.  Rather than radix-sorting 44-60 bit keys over all M pairs,
// the path sorts in two stages that give the same order:
//   1. sort the V*n (view, Gaussian) records by their float32 depth bits
//      (stable, so ties keep index order), digits taken of the bits minus
//      their minimum, the passes above the keys' span skipped on the device;
//   2. emit the pairs in that depth order with key = view * tiles + tile and
//      stable-sort them by that key alone -- ceil(bits/8) passes over M
//      (one packed word per pair when record and key fit 32 bits together).
// A stable sort by tile of a sequence already ordered by (depth, index)
// yields (view, tile, depth, index) order.  Records that touch no tile
// (culled) are dropped first by a stable compaction, so only the visible
// ones are depth-sorted (inputs of at most 2^16 records instead sort the
// culled ones last: the same order with fewer launches).  Both stages use
// one hand-written LSD radix sort of 8-bit digits in three forms by size:
// the whole binning in one CTA (at most 4096 records and 256 lists), one
// look-back kernel per pass (at most 64 chunks of 2048 items), or per-chunk
// counts, their scan and a stable scatter per pass.  The visible and
// instance counts live only on the device; later kernels read them from the
// workspace header, so no host round trip is needed and no block works past
// them.
#include <algorithm>

#include "veg_internal.cuh"

namespace veg {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTileItems = kThreads * kItems;  // 2048 items per radix block
constexpr int64_t kSmallRecords = 1 << 16;      // below: no compaction before the sort

// Number of items to process: a fixed count, or min(*dev, cap).
struct Count {
  int64_t fixed;
  const unsigned long long* dev;
  int64_t cap;
  __device__ __forceinline__ int64_t get() const {
    if (dev == nullptr) return fixed;
    unsigned long long m = *dev;
    return (int64_t)(m < (unsigned long long)cap ? m : (unsigned long long)cap);
  }
};

__device__ __forceinline__ float rcp_approx_f(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Exclusive scan of one value per thread over a 256-thread block.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan256(T x, T* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < 8 ? s_warp[lane] : T(0);
    T wi = w;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < 8) s_warp[lane] = wi - w;
  }
  __syncthreads();
  T r = s_warp[warp] + inc - x;
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// radix sort kernels (u32 keys, u32 values, one 1..8-bit digit per pass)
//
// A pass splits the items into chunks of 2048; a CTA ranks a chunk's items
// among equal digits, stages the chunk in digit order in shared memory and
// writes each digit run out contiguously.  A chunk's start in each digit's
// run comes from one of two places:
//  * a table (three kernels per pass: per-chunk digit counts, their scan
//    along each digit, the scatter) -- for large inputs, where every CTA of
//    a wave would otherwise wait on its neighbours;
//  * a chained scan with decoupled look-back (one kernel per pass, after one
//    histogram of all passes): the CTA takes its chunk by ticket, publishes
//    its per-digit counts, then adds the earlier chunks' published values
//    until it meets an inclusive prefix -- for inputs of a few chunks, where
//    the walks are short and the launches dominate.
// ---------------------------------------------------------------------------

// Chunks of `ITEMS` items per thread of a 256-thread block.
template <int ITEMS = kItems>
__device__ __forceinline__ int chunks_of(int64_t n) {
  return (int)((n + kThreads * ITEMS - 1) / (kThreads * ITEMS));
}

constexpr int kMaxPasses = 4;
struct PassDigits {
  int passes;
  int shift[kMaxPasses];
  int nbits[kMaxPasses];
};

// Key range of a sort (the depth sort: the range of its keys, folded into
// the header by the kernels that write them).  Digits are taken of
// key - key_min, and a pass whose digits are then all zero (its shift at or
// beyond the bit length of key_max - key_min) is an identity and does no
// work.  Such passes form a suffix of the passes.  Null: plain keys, no
// pass skipped.
__device__ __forceinline__ uint32_t range_base(const WsHeader* h) {
  return h ? h->key_min : 0u;
}
__device__ __forceinline__ bool pass_skipped(const WsHeader* h, int shift) {
  if (!h) return false;
  const uint32_t lo = h->key_min, hi = h->key_max;
  return hi <= lo || ((hi - lo) >> shift) == 0u;
}

// The values of a sort whose trailing passes may have been skipped: buffer
// v[q % 2], q = the passes that ran.
struct SortedVals {
  const uint32_t* v[2];
  const WsHeader* krange;
  PassDigits pd;
  __device__ __forceinline__ const uint32_t* get() const {
    int q = 0;
#pragma unroll
    for (int p = 0; p < kMaxPasses; ++p)
      if (p < pd.passes && !pass_skipped(krange, pd.shift[p])) ++q;
    return (q & 1) ? v[1] : v[0];
  }
};

// Folds each lane's key range [kmin, kmax] (empty when kmin > kmax) into the
// header: one atomic pair per warp.  Every lane of the warp must call.
__device__ __forceinline__ void fold_key_range(uint32_t kmin, uint32_t kmax, WsHeader* hdr) {
  kmin = __reduce_min_sync(0xffffffffu, kmin);
  kmax = __reduce_max_sync(0xffffffffu, kmax);
  if ((threadIdx.x & 31) == 0 && kmin <= kmax) {
    atomicMin(&hdr->key_min, kmin);
    atomicMax(&hdr->key_max, kmax);
  }
}

// Look-back word: state in the top two bits (0 not yet published, 1 the
// chunk's own count, 2 the inclusive prefix of chunks 0..c), value below.
constexpr unsigned long long kLbAgg = 1ull << 62;
constexpr unsigned long long kLbInc = 2ull << 62;
constexpr unsigned long long kLbValue = (1ull << 62) - 1ull;
// Polls of a look-back word before a pass gives up and flags a timeout.
constexpr int kLookbackSpins = 1 << 20;
// Largest sort (in 2048-item chunks) that takes the look-back passes.
constexpr int kLookbackMaxChunks = 64;

// Per-chunk digit histograms; hist is [2^nbits][nblocks] (nblocks = the
// chunk capacity), blocks stride over the chunks that hold items.
template <int ITEMS>
__global__ void __launch_bounds__(kThreads)
    radix_hist_kernel(const uint32_t* __restrict__ keys, Count cnt, int shift, int nbits,
                      uint32_t* __restrict__ hist, int nblocks, const WsHeader* krange) {
  pdl_enter();
  __shared__ uint32_t s_hist[256];
  if (pass_skipped(krange, shift)) return;
  const uint32_t kb = range_base(krange);
  const int64_t n = cnt.get();
  const int nch = chunks_of<ITEMS>(n);
  const uint32_t mask = (1u << nbits) - 1u;
  const bool digit = threadIdx.x <= mask;
  for (int b = blockIdx.x; b < nch; b += gridDim.x) {
    s_hist[threadIdx.x] = 0;
    __syncthreads();
    // each thread counts ITEMS consecutive keys, loaded as 16-byte vectors
    // (the key arrays are 256-byte aligned) before any shared-memory update
    const int64_t i0 = (int64_t)b * (kThreads * ITEMS) + (int64_t)threadIdx.x * ITEMS;
    if (i0 + ITEMS <= n) {
      const uint4* src = reinterpret_cast<const uint4*>(keys + i0);
      uint32_t k[ITEMS];
#pragma unroll
      for (int q = 0; q < ITEMS / 4; ++q) {
        const uint4 a = __ldg(src + q);
        k[4 * q] = a.x;
        k[4 * q + 1] = a.y;
        k[4 * q + 2] = a.z;
        k[4 * q + 3] = a.w;
      }
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) atomicAdd(&s_hist[((k[j] - kb) >> shift) & mask], 1u);
    } else {
      for (int j = 0; j < ITEMS; ++j)
        if (i0 + j < n) atomicAdd(&s_hist[((__ldg(&keys[i0 + j]) - kb) >> shift) & mask], 1u);
    }
    __syncthreads();
    if (digit) hist[(int64_t)threadIdx.x * nblocks + b] = s_hist[threadIdx.x];
  }
}

// One block per digit: exclusive scan in place of that digit's per-chunk
// counts (the chunks that hold items), and the digit total.
template <int ITEMS>
__global__ void __launch_bounds__(1024)
    radix_scan_rows_kernel(uint32_t* __restrict__ hist, int nblocks, uint32_t* __restrict__ totals,
                           Count cnt, int shift, const WsHeader* krange) {
  pdl_enter();
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_total;
  if (pass_skipped(krange, shift)) return;
  uint32_t* row = hist + (int64_t)blockIdx.x * nblocks;
  nblocks = chunks_of<ITEMS>(cnt.get());
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t carry = 0;
  for (int base = 0; base < nblocks; base += 1024 * 4) {
    uint32_t v[4];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int i = base + threadIdx.x * 4 + k;
      v[k] = i < nblocks ? row[i] : 0u;
      sum += v[k];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = s_warp[lane];
      uint32_t wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
      }
      s_warp[lane] = wi - w;
      if (lane == 31) s_total = wi;
    }
    __syncthreads();
    uint32_t run = carry + s_warp[warp] + inc - sum;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int i = base + threadIdx.x * 4 + k;
      if (i < nblocks) row[i] = run;
      run += v[k];
    }
    carry += s_total;
    __syncthreads();
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

// Digit histograms of every pass over all n keys, added into ghist
// [passes][256] (zeroed beforehand); also zeroes the first pass's look-back
// words [chunks][256] (each pass zeroes the next one's).
__global__ void __launch_bounds__(kThreads)
    radix_global_hist_kernel(const uint32_t* __restrict__ keys, Count cnt, PassDigits pd,
                             uint32_t* __restrict__ ghist, unsigned long long* __restrict__ look,
                             const WsHeader* krange) {
  pdl_enter();
  __shared__ uint32_t s_hist[kMaxPasses][256];
  const uint32_t kb = range_base(krange);
  const int64_t n = cnt.get();
  const int nch = chunks_of(n);
  for (int p = 0; p < kMaxPasses; ++p) s_hist[p][threadIdx.x] = 0u;
  const int64_t nlook = (int64_t)nch * 256;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < nlook;
       i += (int64_t)gridDim.x * kThreads)
    look[i] = 0ull;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    const uint32_t k = __ldg(&keys[i]) - kb;
#pragma unroll
    for (int p = 0; p < kMaxPasses; ++p)
      if (p < pd.passes) atomicAdd(&s_hist[p][(k >> pd.shift[p]) & ((1u << pd.nbits[p]) - 1u)], 1u);
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < kMaxPasses; ++p)
    if (p < pd.passes && (uint32_t)threadIdx.x < (1u << pd.nbits[p]) && s_hist[p][threadIdx.x])
      atomicAdd(&ghist[p * 256 + threadIdx.x], s_hist[p][threadIdx.x]);
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_volatile_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.volatile.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// One stable pass: rank every item among equal digits of its chunk (warp
// order, then lane order = item order), stage the chunk in digit order in
// shared memory and write each digit run out contiguously.  The chunk's
// start in each digit run is dtot-prefix + hist[digit][chunk] (TABLE; blocks
// stride over the chunks) or found by look-back (blocks loop over tickets,
// so a chunk's predecessors belong to blocks that are already running; a
// look-back not answered within `spins` polls sets FLAG_TIMEOUT in the
// header and stops waiting: the output is then void).  dtot: the digit
// totals of the pass.
template <bool TABLE, int ITEMS>
__global__ void __launch_bounds__(kThreads, ITEMS == 4 ? 6 : 4)
    radix_scatter_kernel(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                         uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, Count cnt,
                         int shift, int nbits, const uint32_t* __restrict__ dtot,
                         const uint32_t* __restrict__ hist, int nblocks,
                         unsigned long long* __restrict__ look, unsigned* __restrict__ ticket,
                         WsHeader* __restrict__ hdr, int spins,
                         unsigned long long* __restrict__ look_next, const WsHeader* krange) {
  pdl_enter();
  __shared__ uint32_t s_whist[8][256];
  __shared__ uint32_t s_dbase[256];
  __shared__ uint32_t s_bstart[256];
  __shared__ uint32_t s_warp[8];
  __shared__ uint32_t s_keys[kThreads * ITEMS];
  __shared__ uint32_t s_vals[kThreads * ITEMS];
  __shared__ int s_chunk;
  if (pass_skipped(krange, shift)) return;  // then so is every later pass
  const uint32_t kb = range_base(krange);
  const int64_t n = cnt.get();
  const int nch = chunks_of<ITEMS>(n);
  if (TABLE && (int)blockIdx.x >= nch) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t mask = (1u << nbits) - 1u;
  const bool digit = (uint32_t)tid <= mask;  // rows of hist and dtot exist for digits only
  // exclusive prefix of the digit totals: each digit's first output position
  const uint32_t dpre = block_exclusive_scan256<uint32_t>(digit ? dtot[tid] : 0u, s_warp);
  if (!TABLE && look_next) {  // the next pass's look-back words (unused during this pass)
    const int64_t nl = (int64_t)nch * 256;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + tid; i < nl; i += (int64_t)gridDim.x * kThreads)
      look_next[i] = 0ull;
  }
  for (int it = 0;; ++it) {
    int b;
    if (TABLE) {
      b = (int)blockIdx.x + it * (int)gridDim.x;
      if (b >= nch) break;  // block-uniform
      if (digit) s_dbase[tid] = dpre + hist[(int64_t)tid * nblocks + b];
    } else if (tid == 0) {
      s_chunk = (int)atomicAdd(ticket, 1u);
    }
#pragma unroll
    for (int w = 0; w < 8; ++w) s_whist[w][tid] = 0;
    __syncthreads();
    if (!TABLE) {
      b = s_chunk;
      if (b >= nch) break;  // block-uniform
    }
    const int64_t base = (int64_t)b * (kThreads * ITEMS);

    uint32_t k[ITEMS], v[ITEMS], r[ITEMS];
    const unsigned lt = lanemask_lt();
    // every load in flight before the ranking (whose warp barriers would
    // otherwise wait for each load in turn)
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const int64_t i = base + warp * (ITEMS * 32) + j * 32 + lane;
      k[j] = i < n ? kin[i] : 0u;
      v[j] = i < n && vin ? vin[i] : 0u;
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      int64_t i = base + warp * (ITEMS * 32) + j * 32 + lane;
      bool valid = i < n;
      uint32_t d = valid ? (((k[j] - kb) >> shift) & mask) : 256u;
      unsigned peers = __match_any_sync(0xffffffffu, d);
      uint32_t before = d < 256u ? s_whist[warp][d] : 0u;
      r[j] = before + __popc(peers & lt);
      __syncwarp();
      if (d < 256u && (peers & lt) == 0) s_whist[warp][d] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, and the chunk's digit count
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      uint32_t c = s_whist[w][tid];
      s_whist[w][tid] = run;
      run += c;
    }
    // the chunk in digit order in shared memory: needs only the chunk's own
    // counts, so the item registers are free before the look-back below
    s_bstart[tid] = block_exclusive_scan256<uint32_t>(run, s_warp);
    __syncthreads();  // every digit's start is read below
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      int64_t i = base + warp * (ITEMS * 32) + j * 32 + lane;
      if (i < n) {
        uint32_t d = ((k[j] - kb) >> shift) & mask;
        uint32_t pos = s_bstart[d] + s_whist[warp][d] + r[j];
        if (pos < (uint32_t)(kThreads * ITEMS)) {  // always, when the counts agree
          s_keys[pos] = k[j];
          s_vals[pos] = v[j];
        }
      }
    }
    if (!TABLE && digit) {
      // publish the count, then add the earlier chunks' counts until an
      // inclusive prefix is met, and publish this chunk's inclusive prefix
      unsigned long long* mine = look + (int64_t)b * 256 + tid;
      st_volatile_u64(mine, kLbAgg | run);
      // the earlier chunks' words are read kWindow at a time (independent
      // loads in flight together), then consumed in order: a count is added
      // and the walk goes on, an inclusive prefix ends it, a word not yet
      // published is polled again
      constexpr int kWindow = 16;
      unsigned long long prefix = 0;
      int left = spins;
      int j = b - 1;
      bool done = j < 0;
      while (!done) {
        unsigned long long w[kWindow];
#pragma unroll
        for (int m = 0; m < kWindow; ++m)
          w[m] = j - m >= 0 ? ld_volatile_u64(look + (int64_t)(j - m) * 256 + tid) : kLbInc;
        int used = 0;
#pragma unroll
        for (int m = 0; m < kWindow; ++m) {
          if (done || used < m) continue;  // stop at the first unpublished word
          const unsigned long long st = w[m] & ~kLbValue;
          if (st == 0ull) continue;
          if (j - m >= 0) prefix += w[m] & kLbValue;
          used = m + 1;
          done = st == kLbInc;
        }
        j -= used;
        if (!done && used < kWindow && --left <= 0) {
          atomicOr(&hdr->flags, FLAG_TIMEOUT);
          break;
        }
      }
      st_volatile_u64(mine, kLbInc | (prefix + run));
      s_dbase[tid] = dpre + (uint32_t)prefix;
    }
    __syncthreads();
    const int cnt_valid = (int)min((int64_t)(kThreads * ITEMS), n - base);
    for (int p = tid; p < cnt_valid; p += kThreads) {
      uint32_t key = s_keys[p];
      uint32_t d = ((key - kb) >> shift) & mask;
      uint32_t g = s_dbase[d] + (uint32_t)p - s_bstart[d];
      kout[g] = key;
      if (vout) vout[g] = s_vals[p];  // keys-only sorts carry no values
    }
    __syncthreads();  // the next chunk reuses the shared arrays (and s_chunk)
  }
}

// ---------------------------------------------------------------------------
// binning kernels
// ---------------------------------------------------------------------------

// Depth keys of all records, culled ones (touching no tile) as 0xffffffff so
// that the stable sort puts them last: the path for small inputs, where one
// launch costs more than sorting the culled records.
__global__ void depth_keys_kernel(const float4* __restrict__ geo, const int32_t* __restrict__ tiles,
                                  int64_t nrec, uint32_t* __restrict__ keys,
                                  uint32_t* __restrict__ vals, WsHeader* __restrict__ hdr) {
  pdl_enter();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t key = 0xffffffffu, kmax = 0u;
  if (i < nrec) {
    key = tiles[i] > 0 ? __float_as_uint(geo[i].z) : 0xffffffffu;
    keys[i] = key;
    vals[i] = (uint32_t)i;
    kmax = key;
  }
  fold_key_range(key, kmax, hdr);
}

// Per-chunk counts of the records that touch a tile (index order).
__global__ void __launch_bounds__(kThreads)
    visible_count_kernel(const int32_t* __restrict__ tiles, int64_t nrec,
                         unsigned long long* __restrict__ bsum) {
  pdl_enter();
  __shared__ unsigned s_warp[8];
  const int64_t base = (int64_t)blockIdx.x * kTileItems + (int64_t)threadIdx.x * kItems;
  unsigned c = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) c += (base + k < nrec && tiles[base + k] > 0) ? 1u : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int w = 0; w < 8; ++w) t += s_warp[w];
    bsum[blockIdx.x] = t;
  }
}

// Stable compaction: the visible records' depth keys and indices, in index
// order, at [0, n_visible).
__global__ void __launch_bounds__(kThreads)
    visible_scatter_kernel(const float4* __restrict__ geo, const int32_t* __restrict__ tiles,
                           int64_t nrec, const unsigned long long* __restrict__ bsum,
                           uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                           WsHeader* __restrict__ hdr) {
  pdl_enter();
  __shared__ unsigned long long s_warp[8];
  const int64_t base = (int64_t)blockIdx.x * kTileItems + (int64_t)threadIdx.x * kItems;
  bool vis[kItems];
  uint32_t dk[kItems];
  unsigned long long c = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    vis[k] = base + k < nrec && tiles[base + k] > 0;
    c += vis[k] ? 1ull : 0ull;
  }
  // the depth loads in flight across the scan's barriers
#pragma unroll
  for (int k = 0; k < kItems; ++k) dk[k] = vis[k] ? __float_as_uint(geo[base + k].z) : 0u;
  unsigned long long run = bsum[blockIdx.x] + block_exclusive_scan256<unsigned long long>(c, s_warp);
  uint32_t kmin = 0xffffffffu, kmax = 0u;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    if (!vis[k]) continue;
    const uint32_t key = dk[k];
    keys[run] = key;
    vals[run] = (uint32_t)(base + k);
    kmin = min(kmin, key);
    kmax = max(kmax, key);
    ++run;
  }
  fold_key_range(kmin, kmax, hdr);
}

// Exclusive scan of per-chunk counts in one block; the total to *total.
__global__ void __launch_bounds__(1024)
    chunk_scan_kernel(unsigned long long* __restrict__ bsum, int nb,
                      unsigned long long* __restrict__ total) {
  pdl_enter();
  __shared__ unsigned long long s_warp[32];
  __shared__ unsigned long long s_total;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long carry = 0;
  for (int base = 0; base < nb; base += 1024) {
    const int i = base + threadIdx.x;
    const unsigned long long x = i < nb ? bsum[i] : 0ull;
    unsigned long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      const unsigned long long w = s_warp[lane];
      unsigned long long wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
      }
      s_warp[lane] = wi - w;
      if (lane == 31) s_total = wi;
    }
    __syncthreads();
    if (i < nb) bsum[i] = carry + s_warp[warp] + inc - x;
    carry += s_total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// Sums of tiles_touched over blocks of 256 records taken in depth order (the
// blocks of the emission kernel).
__global__ void __launch_bounds__(256)
    count_reduce_kernel(const int32_t* __restrict__ tiles, SortedVals sorted, Count cnt,
                        unsigned long long* __restrict__ bsum) {
  pdl_enter();
  const uint32_t* __restrict__ order = sorted.get();
  __shared__ unsigned long long s_warp[8];
  const int64_t nrec = cnt.get();
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  unsigned long long acc = i < nrec ? (unsigned)tiles[order[i]] : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < 8; ++w) t += s_warp[w];
    bsum[blockIdx.x] = t;
  }
}

// Exclusive scan of the block sums (one block of 1024 threads); writes the
// instance total and the capacity flag into the header.
__global__ void __launch_bounds__(1024)
    count_top_kernel(unsigned long long* __restrict__ bsum, int nb, WsHeader* __restrict__ hdr,
                     int64_t capacity) {
  pdl_enter();
  __shared__ unsigned long long s_warp[32];
  __shared__ unsigned long long s_total;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long carry = 0;
  for (int base = 0; base < nb; base += 1024) {
    int i = base + threadIdx.x;
    unsigned long long x = i < nb ? bsum[i] : 0ull;
    unsigned long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      unsigned long long w = s_warp[lane];
      unsigned long long wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
      }
      s_warp[lane] = wi - w;
      if (lane == 31) s_total = wi;
    }
    __syncthreads();
    if (i < nb) bsum[i] = carry + s_warp[warp] + inc - x;
    carry += s_total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    hdr->n_instances = carry;
    if (carry > (unsigned long long)capacity) atomicOr(&hdr->flags, FLAG_CAPACITY);
  }
}

// With rec_bits > 0 (records and list ids fit one 32-bit word together) each
// pair is written as one word, list id << rec_bits | record, into ikeys.
// Writes the (global tile id, record) pairs of 32 consecutive records (in
// depth order) per warp, tiles of a record row-major, below capacity; the
// global id of tile (tx, ty) of view v is vm.tile_off[v] + ty * tiles_x[v]
// + tx.  The
// warp's instances form one contiguous run; lanes write consecutive
// positions of it, each finding the record that owns its position by a
// binary search over the lanes' offsets (offsets increase with the lane).
__global__ void __launch_bounds__(256)
    emit_kernel(const int32_t* __restrict__ tiles, const short4* __restrict__ rect,
                SortedVals sorted, const unsigned long long* __restrict__ bsum, Count visible,
                int64_t n_per_view, ViewMap vm, int64_t capacity, int rec_bits,
                uint32_t* __restrict__ ikeys, uint32_t* __restrict__ ivals) {
  pdl_enter();
  __shared__ unsigned long long s_warp[8];
  const uint32_t* __restrict__ order = sorted.get();
  const int lane = threadIdx.x & 31;
  const int64_t nrec = visible.get();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t g = 0, cnt = 0;
  short4 rc = make_short4(0, 0, 0, 0);
  if (i < nrec) {
    g = order[i];
    cnt = (uint32_t)tiles[g];
    if (cnt) rc = rect[g];
  }
  // the record's first instance: the block's offset (scanned block sums)
  // plus the block's exclusive scan, saturated at 0xffffffff beyond 2^32
  // instances; records past the count get 0xffffffff
  const unsigned long long off64 =
      bsum[blockIdx.x] + block_exclusive_scan256<unsigned long long>(cnt, s_warp);
  const uint32_t off = i < nrec && off64 < 0xffffffffull ? (uint32_t)off64 : 0xffffffffu;
  const uint32_t first = __shfl_sync(0xffffffffu, off, 0);
  unsigned long long end = off == 0xffffffffu ? 0ull : (unsigned long long)off + cnt;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) end = max(end, __shfl_xor_sync(0xffffffffu, end, o));
  if (first == 0xffffffffu || first >= (uint64_t)capacity) return;  // warp-uniform
  const uint32_t stop = (uint32_t)min(end, (unsigned long long)capacity);
  const int wx = rc.z - rc.x;
  const int view = (int)(g / (uint32_t)n_per_view);
  const uint32_t kb = (uint32_t)vm.tile_off[view];
  const int tx_v = vm.tiles_x[view];
  for (uint32_t base = first; base < stop; base += 32) {
    const uint32_t p = base + lane;
    // owner: the largest lane whose offset is <= p
    int lo = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const uint32_t o = __shfl_sync(0xffffffffu, off, lo + step);
      if (o <= p) lo += step;
    }
    const uint32_t o_off = __shfl_sync(0xffffffffu, off, lo);
    const int o_wx = __shfl_sync(0xffffffffu, wx, lo);
    const int o_x0 = __shfl_sync(0xffffffffu, (int)rc.x, lo);
    const int o_y0 = __shfl_sync(0xffffffffu, (int)rc.y, lo);
    const uint32_t o_kb = __shfl_sync(0xffffffffu, kb, lo);
    const int o_tx = __shfl_sync(0xffffffffu, tx_v, lo);
    const uint32_t o_g = __shfl_sync(0xffffffffu, g, lo);
    if (p < stop) {
      const int local = (int)(p - o_off);
      // quotient by a float reciprocal (within one of the floor: local is
      // below the rect's area, at most 1024^2 tiles), corrected to the floor
      int ry = (int)((float)local * rcp_approx_f((float)o_wx));
      int rx = local - ry * o_wx;
      if (rx < 0) {
        --ry;
        rx += o_wx;
      } else if (rx >= o_wx) {
        ++ry;
        rx -= o_wx;
      }
      const uint32_t key = o_kb + (uint32_t)((o_y0 + ry) * o_tx + o_x0 + rx);
      if (rec_bits > 0) {
        ikeys[p] = (key << rec_bits) | o_g;  // one packed word: list id, record
      } else {
        ikeys[p] = key;
        ivals[p] = o_g;
      }
    }
  }
}

// Empties the tile ranges; block 0 also clears the status flags and the
// radix sorts' digit histograms and tickets (`small` words).
__global__ void zero_ranges_kernel(int2* __restrict__ ranges, int64_t count,
                                   uint32_t* __restrict__ small, int nsmall,
                                   WsHeader* __restrict__ hdr) {
  pdl_enter();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) ranges[i] = make_int2(0, 0);
  if (blockIdx.x == 0) {
    for (int k = threadIdx.x; k < nsmall; k += blockDim.x) small[k] = 0u;
    if (threadIdx.x == 0) {
      hdr->flags = 0u;
      hdr->key_min = 0xffffffffu;  // empty range, widened by the depth keys' writers
      hdr->key_max = 0u;
    }
  }
}

// Four sorted keys per thread (one 16-byte load; the key array is 256-byte
// aligned): a run starts where the key differs from its predecessor and
// ends where it differs from its successor.  Keys are < 2^31, so 0xffffffff
// marks "no neighbour".
__global__ void ranges_kernel(const uint32_t* __restrict__ keys, Count cnt,
                              int2* __restrict__ ranges, int key_shift,
                              uint32_t* __restrict__ vals) {
  pdl_enter();
  const int64_t n = cnt.get();
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (i0 >= n) return;
  // packed words (key_shift > 0): the list id above key_shift, the record
  // below it (written to vals); 0xffffffff marks "no neighbour" after the
  // shift (list ids are below 2^31)
  uint32_t w[4];
  if (i0 + 4 <= n) {
    const uint4 q = *reinterpret_cast<const uint4*>(keys + i0);
    w[0] = q.x;
    w[1] = q.y;
    w[2] = q.z;
    w[3] = q.w;
  } else {
#pragma unroll
    for (int t = 0; t < 4; ++t) w[t] = i0 + t < n ? keys[i0 + t] : 0u;
  }
  uint32_t k[6];
  k[0] = i0 > 0 ? keys[i0 - 1] >> key_shift : 0xffffffffu;
#pragma unroll
  for (int t = 0; t < 4; ++t) k[1 + t] = i0 + t < n ? w[t] >> key_shift : 0xffffffffu;
  k[5] = i0 + 4 < n ? keys[i0 + 4] >> key_shift : 0xffffffffu;
  const uint32_t rmask = key_shift > 0 ? (0xffffffffu >> (32 - key_shift)) : 0u;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int64_t i = i0 + t;
    if (i >= n) break;
    const uint32_t kk = k[1 + t];
    if (kk != k[t]) ranges[kk].x = (int)i;
    if (kk != k[2 + t]) ranges[kk].y = (int)(i + 1);
    if (vals) vals[i] = w[t] & rmask;
  }
}

// key = (view << (tb + 32)) | (tile of the view << 32) | depth bits, with tb
// the tile bits of the largest view.
__global__ void keys64_kernel(const uint32_t* __restrict__ tkeys, const uint32_t* __restrict__ vals,
                              Count cnt, const float4* __restrict__ geo, ViewMap vm, int tb,
                              int key_shift, uint64_t* __restrict__ keys64) {
  pdl_enter();
  const int64_t n = cnt.get();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t tk = tkeys[i] >> key_shift;
  uint32_t view = (uint32_t)view_of_tile(vm, (int)tk);
  uint32_t tile = tk - (uint32_t)vm.tile_off[view];
  uint32_t depth = __float_as_uint(geo[vals[i]].z);
  keys64[i] = ((uint64_t)view << (tb + 32)) | ((uint64_t)tile << 32) | (uint64_t)depth;
}

struct Layout {
  WsHeader* hdr;
  uint32_t *dk0, *dv0, *dk1, *dv1;
  unsigned long long* esum;  // instances per 256-record block in depth order, then their scan
  unsigned long long* bsum;
  uint32_t *ik0, *ik1, *iv0;
  uint32_t *hist, *totals;  // table passes: [256][nb_hist] per-chunk counts, [256] totals
  uint32_t* small;  // look-back passes: [2 sorts][kMaxPasses][256] digit totals, then
                    // [2][kMaxPasses] tickets
  unsigned long long* look[2];  // look-back words of alternate passes, [chunks][256] each
  int nb_rec, nb_hist, nb_emit;
  size_t bytes;
};
constexpr int kSmallWords = 2 * kMaxPasses * 256 + 2 * kMaxPasses;

Layout carve(void* ws, int64_t nrec, int64_t capacity) {
  Carver c(ws);
  Layout L;
  L.hdr = c.take<WsHeader>(1);
  L.dk0 = c.take<uint32_t>(nrec);
  L.dv0 = c.take<uint32_t>(nrec);
  L.dk1 = c.take<uint32_t>(nrec);
  L.dv1 = c.take<uint32_t>(nrec);
  L.nb_emit = (int)std::max<int64_t>(1, (nrec + 255) / 256);
  L.esum = c.take<unsigned long long>(L.nb_emit);
  L.nb_rec = (int)std::max<int64_t>(1, (nrec + kTileItems - 1) / kTileItems);
  L.bsum = c.take<unsigned long long>(L.nb_rec);
  L.ik0 = c.take<uint32_t>(capacity);
  L.ik1 = c.take<uint32_t>(capacity);
  L.iv0 = c.take<uint32_t>(capacity);
  // the depth sort's table passes take chunks of 1024 records
  L.nb_hist = (int)std::max<int64_t>(2 * (int64_t)L.nb_rec,
                                     (capacity + kTileItems - 1) / kTileItems);
  L.hist = c.take<uint32_t>((size_t)256 * L.nb_hist);
  L.totals = c.take<uint32_t>(256);
  L.small = c.take<uint32_t>(kSmallWords);
  // look-back words only for the sorts that take the look-back passes
  const int64_t look_chunks = std::min<int64_t>(L.nb_hist, kLookbackMaxChunks);
  L.look[0] = c.take<unsigned long long>((size_t)look_chunks * 256);
  L.look[1] = c.take<unsigned long long>((size_t)look_chunks * 256);
  L.bytes = c.bytes();
  return L;
}

// CTAs of a radix pass: one wave (4 per SM) at most; they take chunks by
// ticket until none is left.
int pass_grid(int nblocks, int per_sm = 4) {
  static std::atomic<int> sms[64];  // per device, 0 until queried
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  int v = sms[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1)
      v = 1;
    sms[dev].store(v, std::memory_order_relaxed);
  }
  return std::max(1, std::min(nblocks, per_sm * v));
}

// The three table kernels of every pass, ITEMS items per thread (chunks of
// 256 ITEMS items; `chunks` of them at most).
template <int ITEMS>
void table_passes(uint32_t* const k[2], uint32_t* const v[2], Count cnt, const PassDigits& pd,
                  int chunks, const Layout& L, const WsHeader* krange, cudaStream_t stream,
                  int spins) {
  const int grid = pass_grid(chunks, ITEMS == 4 ? 6 : 4);  // the scatter's CTAs per SM
  for (int p = 0; p < pd.passes; ++p) {
    const uint32_t* kin = k[p & 1];
    const uint32_t* vin = v[p & 1];
    // the histogram kernel is light (28 registers, 1 KB): twice the blocks
    launch_k(radix_hist_kernel<ITEMS>, std::min(chunks, 2 * grid), kThreads, 0, stream, kin, cnt,
             pd.shift[p], pd.nbits[p], L.hist, chunks, krange);
    launch_k(radix_scan_rows_kernel<ITEMS>, 1 << pd.nbits[p], 1024, 0, stream, L.hist, chunks,
             L.totals, cnt, pd.shift[p], krange);
    launch_k(radix_scatter_kernel<true, ITEMS>, grid, kThreads, 0, stream, kin, vin,
             k[(p + 1) & 1], v[(p + 1) & 1], cnt, pd.shift[p], pd.nbits[p],
             (const uint32_t*)L.totals, (const uint32_t*)L.hist, chunks,
             (unsigned long long*)nullptr, (unsigned*)nullptr, L.hdr, spins,
             (unsigned long long*)nullptr, krange);
  }
  count_launch(3 * pd.passes);
}

// Stable LSD sort of (key, value) pairs by the key bits [base_shift,
// base_shift + bits), in passes of balanced digit widths (at most 8 bits);
// with v[0] and v[1] null the keys alone are sorted.  Buffers ping-pong
// k[p % 2] -> k[(p + 1) % 2]; with `krange` (the depth sort) trailing passes
// over constant digits are skipped on the device, so the result's buffer is
// known there only: the returned SortedVals names it (without `krange`,
// v[passes % 2]).  Up to kLookbackMaxChunks chunks (max_chunks, known on the
// host: the item count itself lives on the device) the passes are
// look-back kernels after one histogram of all passes (`sort`, 0 or 1,
// picks their digit totals and tickets); above, three table kernels per
// pass.
SortedVals radix_sort(uint32_t* const k[2], uint32_t* const v[2], Count cnt, int bits,
                      int max_chunks, const Layout& L, int sort, const WsHeader* krange,
                      cudaStream_t stream, int spins = kLookbackSpins, int base_shift = 0) {
  PassDigits pd;
  pd.passes = std::max(1, (bits + 7) / 8);
  int shift = base_shift;
  for (int p = 0; p < pd.passes; ++p) {
    const int nb = (bits - (shift - base_shift) + (pd.passes - p) - 1) /
                   (pd.passes - p);  // balanced widths
    pd.shift[p] = shift;
    pd.nbits[p] = std::max(1, nb);
    shift += nb;
  }
  SortedVals out{{v[0], v[1]}, krange, pd};
  if (max_chunks > kLookbackMaxChunks) {
    // the depth sort (about one item per Gaussian, L2-resident) in chunks of
    // 1024: twice the CTAs, each with half the ranking chain; the tile sort
    // in chunks of 2048
    if (sort == 0)
      table_passes<4>(k, v, cnt, pd, 2 * max_chunks, L, krange, stream, spins);
    else
      table_passes<8>(k, v, cnt, pd, max_chunks, L, krange, stream, spins);
    return out;
  }
  const int grid = pass_grid(max_chunks);
  uint32_t* ghist = L.small + sort * kMaxPasses * 256;
  unsigned* tickets = L.small + 2 * kMaxPasses * 256 + sort * kMaxPasses;
  launch_k(radix_global_hist_kernel, grid, kThreads, 0, stream, (const uint32_t*)k[0], cnt, pd,
           ghist, L.look[0], krange);
  for (int p = 0; p < pd.passes; ++p)
    launch_k(radix_scatter_kernel<false, kItems>, grid, kThreads, 0, stream,
             (const uint32_t*)k[p & 1],
             (const uint32_t*)v[p & 1], k[(p + 1) & 1], v[(p + 1) & 1], cnt, pd.shift[p],
             pd.nbits[p], (const uint32_t*)(ghist + p * 256), (const uint32_t*)nullptr, 0,
             L.look[p & 1], tickets + p, L.hdr, spins,
             p + 1 < pd.passes ? L.look[(p + 1) & 1] : (unsigned long long*)nullptr, krange);
  count_launch(1 + pd.passes);
  return out;
}

inline unsigned grid_for(int64_t n, int threads) {
  return (unsigned)std::max<int64_t>(1, (n + threads - 1) / threads);
}

}  // namespace

size_t binsort_ws_bytes(int64_t n, int n_views, int64_t capacity) {
  return carve(nullptr, n * n_views, capacity).bytes;
}

namespace {

// ---------------------------------------------------------------------------
// One-CTA binning for small inputs (at most kOneCtaRecords records and
// kOneCtaLists tile lists): the whole path of the kernels above in one
// launch of 1024 threads, with the records in shared memory.  Same output,
// bit for bit: the visible records in index order, their stable radix sort
// by depth bits (passes above the keys' span skipped), the instance offsets
// in depth order, then the stable sort of the first `capacity` instances by
// list as a counting sort: each warp owns a contiguous run of 128 sorted
// records, counts its instances per list, and after a scan over (list,
// warp) writes them at their places in emission order.  Every warp
// collective sits in a loop whose trip count is the same for all lanes of
// the warp.
// ---------------------------------------------------------------------------

constexpr int kOneCtaThreads = 1024;
constexpr int kOneCtaWarps = kOneCtaThreads / 32;
constexpr int kOneCtaRecords = 4096;                    // 4 per thread, 128 per warp
constexpr int kOneCtaLists = 256;
constexpr int kOneCtaPerWarp = kOneCtaRecords / kOneCtaWarps;

struct OneCtaSmem {
  uint32_t key[2][kOneCtaRecords];
  uint32_t rec[2][kOneCtaRecords];
  uint32_t off[kOneCtaRecords + 1];            // instance offsets of the sorted records
  uint32_t lbase[kOneCtaRecords];              // list of each sorted record's first tile
  uint32_t shape[kOneCtaRecords];              // its rect width | view's tiles_x << 16
  uint16_t wcnt[kOneCtaWarps][256];           // per warp: digit counts, then list counts
  uint32_t lmask[kOneCtaWarps][kOneCtaLists];  // per warp and list: lanes touching the list
  uint32_t lstart[kOneCtaLists];               // first instance of each list
  uint32_t ltotal[kOneCtaLists];
  uint32_t scan[kOneCtaWarps];
  uint32_t kmin, kmax, nvis;
};

// Exclusive scan of one value per thread over the 1024-thread block; the
// total to *total (read after the call's last barrier).
__device__ __forceinline__ uint32_t onecta_scan(uint32_t x, uint32_t* s_warp, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = s_warp[lane];
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    s_warp[lane] = wi - w;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  const uint32_t r = s_warp[warp] + inc - x;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kOneCtaThreads, 1)
    bin_one_cta_kernel(const float4* __restrict__ geo, const int32_t* __restrict__ tiles,
                       const short4* __restrict__ rect, int nrec, int64_t n_per_view, ViewMap vm,
                       int nlists, int64_t capacity, int tb, uint64_t* __restrict__ keys,
                       uint32_t* __restrict__ vals, int2* __restrict__ ranges,
                       WsHeader* __restrict__ hdr) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char onecta_raw[];
  OneCtaSmem& S = *reinterpret_cast<OneCtaSmem*>(onecta_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lt = lanemask_lt();
  if (tid == 0) {
    S.kmin = 0xffffffffu;
    S.kmax = 0u;
  }
  // 1. the visible records in index order (4 consecutive records per thread)
  uint32_t vis[4], key[4];
  uint32_t c = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = tid * 4 + k;
    vis[k] = i < nrec && tiles[i] > 0;
    key[k] = vis[k] ? __float_as_uint(geo[i].z) : 0u;
    c += vis[k];
  }
  uint32_t kmin = 0xffffffffu, kmax = 0u;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (vis[k]) {
      kmin = min(kmin, key[k]);
      kmax = max(kmax, key[k]);
    }
  kmin = __reduce_min_sync(0xffffffffu, kmin);
  kmax = __reduce_max_sync(0xffffffffu, kmax);
  __syncthreads();  // S.kmin / S.kmax initialised
  if (lane == 0) {
    atomicMin(&S.kmin, kmin);
    atomicMax(&S.kmax, kmax);
  }
  uint32_t pos = onecta_scan(c, S.scan, &S.nvis);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (vis[k]) {
      S.key[0][pos] = key[k];
      S.rec[0][pos] = (uint32_t)(tid * 4 + k);
      ++pos;
    }
  __syncthreads();
  const int nvis = (int)S.nvis;
  const uint32_t kb = S.kmin;
  const uint32_t span = S.kmax > S.kmin ? S.kmax - S.kmin : 0u;

  // 2. stable LSD sort by (key - kmin), 8-bit digits, passes within the span
  int cur = 0;
  for (int shift = 0; shift < 32 && (span >> shift) != 0u; shift += 8) {
    for (int e = tid; e < kOneCtaWarps * 256; e += kOneCtaThreads)
      S.wcnt[e >> 8][e & 255] = 0;
    __syncthreads();
    uint32_t d[4], r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = warp * kOneCtaPerWarp + j * 32 + lane;
      d[j] = i < nvis ? ((S.key[cur][i] - kb) >> shift) & 255u : 256u;
      const unsigned peers = __match_any_sync(0xffffffffu, d[j]);
      const uint32_t before = d[j] < 256u ? S.wcnt[warp][d[j]] : 0u;
      r[j] = before + __popc(peers & lt);
      __syncwarp();
      if (d[j] < 256u && (peers & lt) == 0u)
        S.wcnt[warp][d[j]] = (uint16_t)(before + __popc(peers));
      __syncwarp();
    }
    __syncthreads();
    // per digit: prefix over warps, then over digits
    uint32_t run = 0;
    if (tid < 256)
      for (int w = 0; w < kOneCtaWarps; ++w) {
        const uint32_t x = S.wcnt[w][tid];
        S.wcnt[w][tid] = (uint16_t)run;
        run += x;
      }
    uint32_t unused;
    const uint32_t dstart = onecta_scan(tid < 256 ? run : 0u, S.scan, &unused);
    if (tid < 256) S.lstart[tid] = dstart;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = warp * kOneCtaPerWarp + j * 32 + lane;
      if (d[j] < 256u) {
        const uint32_t q = S.lstart[d[j]] + S.wcnt[warp][d[j]] + r[j];
        if (q < (uint32_t)kOneCtaRecords) {  // always, when the counts agree
          S.key[cur ^ 1][q] = S.key[cur][i];
          S.rec[cur ^ 1][q] = S.rec[cur][i];
        }
      }
    }
    __syncthreads();
    cur ^= 1;
  }
  const uint32_t* order = S.rec[cur];

  // 3. instance offsets in depth order (4 consecutive sorted records per
  //    thread), and each record's list geometry, gathered once
  uint32_t cnt[4], sum = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int j = tid * 4 + k;
    cnt[k] = 0u;
    if (j < nvis) {
      const uint32_t g = order[j];
      const short4 rc = rect[g];
      const int view = (int)(g / (uint32_t)n_per_view);
      const int tx = vm.tiles_x[view];
      cnt[k] = (uint32_t)tiles[g];
      S.lbase[j] = (uint32_t)(vm.tile_off[view] + rc.y * tx + rc.x);
      S.shape[j] = (uint32_t)(rc.z - rc.x) | ((uint32_t)tx << 16);
    }
    sum += cnt[k];
  }
  uint32_t total;
  {
    uint32_t o = onecta_scan(sum, S.scan, &S.off[kOneCtaRecords]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      S.off[tid * 4 + k] = o;
      o += cnt[k];
    }
  }
  __syncthreads();
  total = S.off[kOneCtaRecords];
  const uint32_t m_cap = (uint32_t)min((int64_t)total, capacity);
  if (tid == 0) {
    hdr->n_instances = total;
    hdr->n_visible = (unsigned long long)nvis;
    hdr->flags = (int64_t)total > capacity ? FLAG_CAPACITY : 0u;
  }

  // 4. the first m_cap instances sorted by list.  Warp w owns the sorted
  //    records [128 w, 128 w + 128), 32 at a time, one per lane.  A record
  //    adds at most one instance to a list, so a lane's place among its
  //    round's instances of list l is the number of lower lanes whose
  //    record touches l too: each lane sets its bit in the warp's mask of
  //    every list it touches (shared memory), then reads the masks.  The
  //    lowest lane of a mask adds its count and clears it.  Only __syncwarp
  //    sits between the lanes' own loops.
  for (int e = tid; e < kOneCtaWarps * kOneCtaLists; e += kOneCtaThreads) {
    S.wcnt[e / kOneCtaLists][e % kOneCtaLists] = 0;
    S.lmask[e / kOneCtaLists][e % kOneCtaLists] = 0u;
  }
  __syncthreads();
  const uint32_t bit = 1u << lane;
  for (int pass = 0; pass < 2; ++pass) {  // count, then place
    if (pass == 1) {
      // per list: prefix over warps, then the lists' starts
      uint32_t lrun = 0;
      if (tid < nlists)
        for (int w = 0; w < kOneCtaWarps; ++w) {
          const uint32_t x = S.wcnt[w][tid];
          S.wcnt[w][tid] = (uint16_t)lrun;
          lrun += x;
        }
      uint32_t unused;
      const uint32_t ls = onecta_scan(tid < nlists ? lrun : 0u, S.scan, &unused);
      if (tid < nlists) {
        S.lstart[tid] = ls;
        S.ltotal[tid] = lrun;
      }
      __syncthreads();
    }
    for (int round = 0; round < kOneCtaPerWarp / 32; ++round) {
      const int j = warp * kOneCtaPerWarp + round * 32 + lane;
      int ntk = 0;
      uint32_t lb = 0, g = 0;
      int wx = 1, tx = 0;
      if (j < nvis) {
        const uint32_t e0 = S.off[j];
        const uint32_t e1 = min(S.off[j + 1], m_cap);
        ntk = e1 > e0 ? (int)(e1 - e0) : 0;
        lb = S.lbase[j];
        wx = (int)(S.shape[j] & 0xffffu);
        tx = (int)(S.shape[j] >> 16);
        g = order[j];
      }
      // the record's lists, tiles row-major: lb + ry * tx + rx
      for (int t = 0, rx = 0, ry = 0; t < ntk; ++t) {
        atomicOr(&S.lmask[warp][lb + ry * tx + rx], bit);
        if (++rx == wx) rx = 0, ++ry;
      }
      __syncwarp();
      if (pass == 1) {
        for (int t = 0, rx = 0, ry = 0; t < ntk; ++t) {
          const uint32_t l = lb + (uint32_t)(ry * tx + rx);
          const uint32_t q = S.lstart[l] + S.wcnt[warp][l] + __popc(S.lmask[warp][l] & lt);
          if (q < m_cap) {  // always, when the counts agree
            vals[q] = g;
            if (keys) {
              const uint32_t view = (uint32_t)view_of_tile(vm, (int)l);
              const uint32_t tile = l - (uint32_t)vm.tile_off[view];
              keys[q] = ((uint64_t)view << (tb + 32)) | ((uint64_t)tile << 32) |
                        (uint64_t)__float_as_uint(geo[g].z);
            }
          }
          if (++rx == wx) rx = 0, ++ry;
        }
        __syncwarp();
      }
      for (int t = 0, rx = 0, ry = 0; t < ntk; ++t) {
        const uint32_t l = lb + (uint32_t)(ry * tx + rx);
        const uint32_t m = S.lmask[warp][l];
        if ((m & lt) == 0u) {  // the lowest lane of the list's mask
          S.wcnt[warp][l] = (uint16_t)(S.wcnt[warp][l] + __popc(m));
          S.lmask[warp][l] = 0u;
        }
        if (++rx == wx) rx = 0, ++ry;
      }
      __syncwarp();
    }
    __syncthreads();
  }
  // 5. the ranges of every list
  for (int l = tid; l < nlists; l += kOneCtaThreads)
    ranges[l] = S.ltotal[l] ? make_int2((int)S.lstart[l], (int)(S.lstart[l] + S.ltotal[l]))
                            : make_int2(0, 0);
}

}  // namespace

veg_status binsort_launch(const veg_camera* cams, int n_views, int64_t n, const float4* geo,
                          const int32_t* tiles, const short4* rect, void* ws, int64_t capacity,
                          uint64_t* keys, uint32_t* vals, int2* ranges, cudaStream_t stream) {
  const ViewMap vm = make_viewmap(cams, n_views, 1);
  const int64_t nrec = n * n_views;
  const int64_t nranges = vm.tile_off[n_views];
  Layout L = carve(ws, nrec, capacity);

  // small inputs: the whole binning in one CTA
  if (nrec >= 1 && nrec <= kOneCtaRecords && nranges <= kOneCtaLists) {
    static SmemRecord one_cta;
    if (prepare_smem(bin_one_cta_kernel, sizeof(OneCtaSmem), one_cta, true) == VEG_OK) {
      launch_k(bin_one_cta_kernel, 1, kOneCtaThreads, sizeof(OneCtaSmem), stream, geo, tiles,
               rect, (int)nrec, n, vm, (int)nranges, capacity, tile_bits_of(vm.max_tiles), keys,
               vals, ranges, L.hdr);
      count_launch();
      return launch_status();
    }
  }
  launch_k(zero_ranges_kernel, grid_for(nranges, 256), 256, 0, stream, ranges, nranges, L.small,
           kSmallWords, L.hdr);
  count_launch();
  if (nrec == 0) {
    cudaMemsetAsync(L.hdr, 0, sizeof(WsHeader), stream);
    return launch_status();
  }
  // 1. the visible records (touching a tile) in index order, then their
  //    depth sort; small inputs sort every record with culled ones last
  //    (same order, fewer launches)
  Count cr{0, &L.hdr->n_visible, nrec};
  if (nrec <= kSmallRecords) {
    launch_k(depth_keys_kernel, grid_for(nrec, 256), 256, 0, stream, geo, tiles, nrec, L.dk0, L.dv0,
             L.hdr);
    count_launch();
    cr = Count{nrec, nullptr, 0};
  } else {
    launch_k(visible_count_kernel, L.nb_rec, kThreads, 0, stream, tiles, nrec, L.bsum);
    launch_k(chunk_scan_kernel, 1, 1024, 0, stream, L.bsum, L.nb_rec, &L.hdr->n_visible);
    launch_k(visible_scatter_kernel, L.nb_rec, kThreads, 0, stream, geo, tiles, nrec, L.bsum, L.dk0,
             L.dv0, L.hdr);
    count_launch(3);
  }
  // (the passes above the depth keys' span are skipped on the device)
  uint32_t* const dk[2] = {L.dk0, L.dk1};
  uint32_t* const dv[2] = {L.dv0, L.dv1};
  const SortedVals order = radix_sort(dk, dv, cr, 32, L.nb_rec, L, 0, L.hdr, stream);
  // 2. instance offsets in depth order, total into the header
  launch_k(count_reduce_kernel, L.nb_emit, 256, 0, stream, tiles, order, cr, L.esum);
  launch_k(count_top_kernel, 1, 1024, 0, stream, L.esum, L.nb_emit, L.hdr, capacity);
  count_launch(2);
  // 3. emit (tile key, record) pairs, then stable sort by tile key.  When
  //    record indices and list ids fit one 32-bit word together, each pair
  //    is one packed word and the sort moves keys only (half the bytes);
  //    the ranges kernel then writes the records into vals.
  int bits = 1;
  while (((int64_t)1 << bits) < nranges) ++bits;
  int rec_bits = 1;
  while (((int64_t)1 << rec_bits) < nrec) ++rec_bits;
  const bool packed = rec_bits + bits <= 32;
  if (!packed) rec_bits = 0;
  const int passes = (bits + 7) / 8;
  uint32_t* kbuf[2] = {L.ik0, L.ik1};
  uint32_t* vbuf[2] = {nullptr, nullptr};
  if (!packed) {
    vbuf[passes % 2 == 0 ? 0 : 1] = vals;
    vbuf[passes % 2 == 0 ? 1 : 0] = L.iv0;
  }
  launch_k(emit_kernel, L.nb_emit, 256, 0, stream, tiles, rect, order,
           (const unsigned long long*)L.esum, cr, n, vm, capacity, rec_bits, kbuf[0], vbuf[0]);
  count_launch();
  Count ci{0, &L.hdr->n_instances, capacity};
  const int nb_inst = (int)std::max<int64_t>(1, (capacity + kTileItems - 1) / kTileItems);
  radix_sort(kbuf, vbuf, ci, bits, nb_inst, L, 1, nullptr, stream, kLookbackSpins, rec_bits);
  const uint32_t* fkeys = kbuf[passes & 1];
  // 4. per-tile ranges (and the records, from packed words) and optional
  //    64-bit keys
  launch_k(ranges_kernel, grid_for(capacity, 1024), 256, 0, stream, fkeys, ci, ranges, rec_bits,
           packed ? vals : (uint32_t*)nullptr);
  count_launch();
  if (keys) {
    launch_k(keys64_kernel, grid_for(capacity, 256), 256, 0, stream, fkeys, vals, ci, geo, vm,
             tile_bits_of(vm.max_tiles), rec_bits, keys);
    count_launch();
  }
  return launch_status();
}

namespace {

// Longest-first order of the tiles (one CTA): tiles are bucketed by
// floor(log2(list length)) and the buckets emitted from the longest down,
// empty tiles last.  Order inside a bucket is unspecified; it only steers
// the CTA schedule, never a result.
__global__ void __launch_bounds__(1024)
    tile_order_kernel(const int2* __restrict__ ranges, int count, int32_t* __restrict__ order) {
  pdl_enter();
  __shared__ unsigned s_cnt[33];
  __shared__ unsigned s_off[33];
  if (threadIdx.x < 33) s_cnt[threadIdx.x] = 0u;
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const int2 r = ranges[i];
    const unsigned len = (unsigned)(r.y - r.x);
    atomicAdd(&s_cnt[len ? 32 - __clz(len) : 0], 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned off = 0;
    for (int b = 32; b >= 0; --b) {
      s_off[b] = off;
      off += s_cnt[b];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const int2 r = ranges[i];
    const unsigned len = (unsigned)(r.y - r.x);
    order[atomicAdd(&s_off[len ? 32 - __clz(len) : 0], 1u)] = i;
  }
}

}  // namespace

veg_status tile_order_launch(const int2* ranges, int count, int32_t* order, cudaStream_t stream) {
  if (count == 0) return VEG_OK;
  launch_k(tile_order_kernel, 1, 1024, 0, stream, ranges, count, order);
  count_launch();
  return launch_status();
}

}  // namespace veg

extern "C" veg_status veg_tile_order(const int32_t* tile_ranges, int64_t count,
                                     int32_t* tile_order, cudaStream_t stream) {
  if (count < 0 || count >= ((int64_t)1 << 31) || (count > 0 && (!tile_ranges || !tile_order)) ||
      (reinterpret_cast<uintptr_t>(tile_ranges) & 7))
    return VEG_ERR_INVALID_ARGUMENT;
  return veg::tile_order_launch(reinterpret_cast<const int2*>(tile_ranges), (int)count,
                                tile_order, stream);
}

extern "C" veg_status veg_bin_sort_workspace_size(int64_t n, int32_t n_views, int64_t capacity,
                                                  int32_t width, int32_t height, size_t* bytes) {
  if (!bytes || n < 0 || n_views < 1 || n_views > VEG_MAX_VIEWS || capacity < 0 ||
      capacity >= ((int64_t)1 << 31) || width < 1 || height < 1 || width > VEG_MAX_IMAGE ||
      height > VEG_MAX_IMAGE)
    return VEG_ERR_INVALID_ARGUMENT;
  *bytes = veg::binsort_ws_bytes(n, n_views, capacity);
  return VEG_OK;
}

extern "C" veg_status veg_bin_sort(const veg_camera* cams, int32_t n_views, int64_t n,
                                   const float* splat_geo, const int32_t* tiles_touched,
                                   const int16_t* rect, void* workspace, size_t workspace_bytes,
                                   int64_t capacity, uint64_t* keys, uint32_t* vals,
                                   int32_t* tile_ranges, cudaStream_t stream) {
  using namespace veg;
  veg_status st = check_cameras(cams, n_views);
  if (st != VEG_OK) return st;
  if (n < 0 || capacity < 0 || capacity >= ((int64_t)1 << 31) || !workspace || !tile_ranges ||
      (capacity > 0 && !vals) || (n > 0 && (!splat_geo || !tiles_touched || !rect)))
    return VEG_ERR_INVALID_ARGUMENT;
  if (n * n_views >= ((int64_t)1 << 31)) return VEG_ERR_INVALID_ARGUMENT;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) || !aligned16(splat_geo) ||
      (reinterpret_cast<uintptr_t>(rect) & 7) || (reinterpret_cast<uintptr_t>(tile_ranges) & 7))
    return VEG_ERR_INVALID_ARGUMENT;
  if (total_tiles_of(cams, n_views) >= ((int64_t)1 << 31)) return VEG_ERR_INVALID_ARGUMENT;
  if (workspace_bytes < binsort_ws_bytes(n, n_views, capacity))
    return VEG_ERR_INVALID_ARGUMENT;
  return binsort_launch(cams, n_views, n, reinterpret_cast<const float4*>(splat_geo),
                        tiles_touched, reinterpret_cast<const short4*>(rect), workspace, capacity,
                        keys, vals, reinterpret_cast<int2*>(tile_ranges), stream);
}

extern "C" veg_status veg_sync_status(const void* workspace, cudaStream_t stream,
                                      int64_t* n_instances) {
  if (!workspace) return VEG_ERR_INVALID_ARGUMENT;
  veg::WsHeader h;
  if (cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
    return VEG_ERR_CUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return VEG_ERR_CUDA;
  if (n_instances) *n_instances = (int64_t)h.n_instances;
  if (h.flags & veg::FLAG_TIMEOUT) return VEG_ERR_TIMEOUT;
  return (h.flags & veg::FLAG_CAPACITY) ? VEG_ERR_CAPACITY : VEG_OK;
}

// ---------------------------------------------------------------------------
// A check of the radix passes' bounded waits on the device.
// ---------------------------------------------------------------------------

namespace veg {
namespace {

// Seeded keys (a multiplicative hash of the index, with repeats) and their
// indices; with `starve`, pass 0's first ticket is taken in advance so that
// chunk 0 is never sorted and never published.
__global__ void lookback_check_keys_kernel(uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                           int64_t n, unsigned* __restrict__ ticket0, int starve) {
  pdl_enter();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    keys[i] = ((uint32_t)i * 2654435761u) >> 4;
    vals[i] = (uint32_t)i;
  }
  if (i == 0 && starve) *ticket0 = 1u;
}

}  // namespace
}  // namespace veg

extern "C" veg_status veg_radix_lookback_check(void* workspace, size_t workspace_bytes, int64_t n,
                                               int32_t starve_first, int32_t spins,
                                               uint32_t* keys_out, uint32_t* vals_out,
                                               cudaStream_t stream) {
  using namespace veg;
  if (!workspace || n < 1 || n > (int64_t)kLookbackMaxChunks * kTileItems || spins < 1 ||
      !keys_out || !vals_out || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return VEG_ERR_INVALID_ARGUMENT;
  Layout L = carve(workspace, n, 0);
  if (workspace_bytes < L.bytes) return VEG_ERR_INVALID_ARGUMENT;
  if (cudaMemsetAsync(L.hdr, 0, sizeof(WsHeader), stream) != cudaSuccess ||
      cudaMemsetAsync(L.small, 0, kSmallWords * sizeof(uint32_t), stream) != cudaSuccess)
    return VEG_ERR_CUDA;
  launch_k(lookback_check_keys_kernel, grid_for(n, 256), 256, 0, stream, L.dk0, L.dv0, n,
           L.small + 2 * kMaxPasses * 256, (int)(starve_first != 0));
  count_launch();
  uint32_t* const dk[2] = {L.dk0, L.dk1};
  uint32_t* const dv[2] = {L.dv0, L.dv1};
  radix_sort(dk, dv, Count{n, nullptr, 0}, 32, L.nb_rec, L, 0, nullptr, stream,
             spins);  // 4 passes: into dk0, dv0
  if (cudaMemcpyAsync(keys_out, L.dk0, (size_t)n * 4, cudaMemcpyDeviceToDevice, stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(vals_out, L.dv0, (size_t)n * 4, cudaMemcpyDeviceToDevice, stream) !=
          cudaSuccess)
    return VEG_ERR_CUDA;
  return launch_status();
}

// ---------------------------------------------------------------------------
// Allocation-free binning: the same kernels with their scratch in a fixed
// device array instead of a caller workspace.
// ---------------------------------------------------------------------------

#include <cuda.h>  // driver types only; the functions are resolved at run time

#include <mutex>

namespace veg {
namespace {

// 16 MiB of scratch held by every GPU that loads the library, until exit.
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;
constexpr int kMaxDevices = 64;

// Address of the array per device, valid for the context it was looked up
// in: a device reset (or a primary context released and created again)
// reloads the library's module, and the array may then sit elsewhere.
struct StaticScratch {
  unsigned long long ctx_id;  // cuCtxGetId of the context, 0 = not looked up
  void* ptr;
};
std::mutex g_static_mu;
StaticScratch g_static[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current context (the library links no
// driver library: both driver functions are resolved through the runtime).
veg_status current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (get_current == nullptr || get_id == nullptr) {
    void* f0 = nullptr;
    void* f1 = nullptr;
    cudaDriverEntryPointQueryResult q0, q1;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault,
                                         &q0) != cudaSuccess ||
        q0 != cudaDriverEntryPointSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || f0 == nullptr || f1 == nullptr)
      return VEG_ERR_CUDA;
    get_current = reinterpret_cast<CtxGetCurrentFn>(f0);
    get_id = reinterpret_cast<CtxGetIdFn>(f1);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return VEG_ERR_CUDA;
  if (get_id(ctx, id) != CUDA_SUCCESS || *id == 0) return VEG_ERR_CUDA;
  return VEG_OK;
}

}  // namespace
}  // namespace veg

static __device__ __align__(256) unsigned char g_binsort_scratch[veg::kStaticScratchBytes];

// The array's name is only a host-side handle: its device address is looked
// up with the device current, once per context.  A lookup is refused while
// `stream` is being captured (it would run inside the caller's capture).
static veg_status static_scratch_address(cudaStream_t stream, void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return VEG_ERR_CUDA;
  if (dev < 0 || dev >= veg::kMaxDevices) return VEG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(veg::g_static_mu);
  unsigned long long ctx = 0;
  if (veg::current_context_id(&ctx) != VEG_OK) {
    // no context current on this thread yet: make the device's primary
    // context current (the runtime creates it; nothing is allocated)
    if (cudaSetDevice(dev) != cudaSuccess) return VEG_ERR_CUDA;
    veg_status st = veg::current_context_id(&ctx);
    if (st != VEG_OK) return st;
  }
  veg::StaticScratch& e = veg::g_static[dev];
  if (e.ctx_id != ctx || e.ptr == nullptr) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess ||
        cap != cudaStreamCaptureStatusNone) {
      cudaGetLastError();  // an implicit-capture error is not the caller's
      return VEG_ERR_UNSUPPORTED;
    }
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_binsort_scratch) != cudaSuccess || p == nullptr)
      return VEG_ERR_CUDA;
    e.ptr = p;
    e.ctx_id = ctx;
  }
  *out = e.ptr;
  return VEG_OK;
}

extern "C" veg_status veg_bin_sort_static(const veg_camera* cams, int32_t n_views, int64_t n,
                                          const float* splat_geo, const int32_t* tiles_touched,
                                          const int16_t* rect, int64_t capacity, uint64_t* keys,
                                          uint32_t* vals, int32_t* tile_ranges,
                                          int64_t* n_instances, cudaStream_t stream) {
  using namespace veg;
  veg_status st = check_cameras(cams, n_views);
  if (st != VEG_OK) return st;
  if (n < 0 || capacity < 0 || capacity >= ((int64_t)1 << 31) || !tile_ranges ||
      (capacity > 0 && !vals) || (n > 0 && (!splat_geo || !tiles_touched || !rect)))
    return VEG_ERR_INVALID_ARGUMENT;
  if (n * n_views >= ((int64_t)1 << 31)) return VEG_ERR_INVALID_ARGUMENT;
  if (!aligned16(splat_geo) || (reinterpret_cast<uintptr_t>(rect) & 7) ||
      (reinterpret_cast<uintptr_t>(tile_ranges) & 7) ||
      (reinterpret_cast<uintptr_t>(n_instances) & 7))
    return VEG_ERR_INVALID_ARGUMENT;
  if (total_tiles_of(cams, n_views) >= ((int64_t)1 << 31)) return VEG_ERR_INVALID_ARGUMENT;
  if (binsort_ws_bytes(n, n_views, capacity) > kStaticScratchBytes)
    return VEG_ERR_UNSUPPORTED;
  void* ws = nullptr;
  st = static_scratch_address(stream, &ws);
  if (st != VEG_OK) return st;
  st = binsort_launch(cams, n_views, n, reinterpret_cast<const float4*>(splat_geo),
                      tiles_touched, reinterpret_cast<const short4*>(rect), ws, capacity, keys,
                      vals, reinterpret_cast<int2*>(tile_ranges), stream);
  if (st != VEG_OK) return st;
  if (n_instances &&
      cudaMemcpyAsync(n_instances, &static_cast<WsHeader*>(ws)->n_instances, sizeof(int64_t),
                      cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
    return VEG_ERR_CUDA;
  return VEG_OK;
}
