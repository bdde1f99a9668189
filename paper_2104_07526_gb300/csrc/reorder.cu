// Vertex-order kernels (Sec. 4, and the orderings listed in Sec. 5):
// bounds, 30-bit and 63-bit Morton codes, a stable LSD radix sort of (32-bit
// key, 32-bit index) pairs whose last pass moves the point records to their
// final positions, and the 128-point batch shuffle.  A 63-bit code sorts as
// two 32-bit halves: the low half first (the high half carried along), then
// the high half, both stable, which is a stable sort by the whole code.
//
// Radix sort: 8-bit digits, one pass per digit, three steps per pass:
//   1. k_sort_hist: per tile of 6144 keys (5120 in the random shuffle,
//      whose passes carry records), count each digit (the first
//      pass's counts come from the kernel that made the keys);
//   2. exclusive scan of the counts in digit-major order, which gives every
//      (digit, tile) its first output slot;
//   3. k_sort_scatter: each warp of a tile takes 768 (640) consecutive keys and
//      counts their digits (per 32 keys, one match.any when their digits
//      form few runs, else eight ballots, one per digit bit);
//      one prefix over (digit, warp) then gives every warp its first slot
//      per digit, and the warp ranks its keys again in index order into the
//      tile's digit-sorted order in shared memory.  The tile is then written
//      out run by run, so each digit's keys leave as one contiguous,
//      coalesced run.
// Ranks follow index order, so each pass, and the sort, is stable.
#include <cstdint>
#include <mutex>
#include <type_traits>

#include "../../include/pcr.h"
#include "common.cuh"
#include "launch.h"

namespace pcr {

namespace {

// Debug builds (PCR_DEBUG) check every gathered index and every scatter
// destination against the cloud before the access; a failure sets
// PCR_DEVICE_ERROR_BOUNDS in this file's error word (read by
// pcr_last_device_error) and skips the access.  Release builds check nothing.
#ifdef PCR_DEBUG
__device__ uint32_t g_reorder_error_word;
#endif
__device__ __forceinline__ bool debug_in_range(uint64_t i, uint64_t n) {
#ifdef PCR_DEBUG
  if (i >= n) {
    atomicOr(&g_reorder_error_word, static_cast<uint32_t>(PCR_DEVICE_ERROR_BOUNDS));
    return false;
  }
#else
  (void)i;
  (void)n;
#endif
  return true;
}

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 24;  // keys per lane in a tile (Morton codes, batch keys)
constexpr uint32_t kTile = kSortThreads * kSortRounds;
// The random shuffle's sort carries 16-byte records: tiles of 20 keys per
// lane keep each block's record window smaller (800M shuffle 34.4 ms with
// 24, 30.6 with 20, 30.9 with 16).
constexpr int kShuffleRounds = 20;
constexpr int kMinRounds = kShuffleRounds < kSortRounds ? kShuffleRounds : kSortRounds;
template <int ROUNDS>
constexpr uint32_t kTileOf = kSortThreads * ROUNDS;
constexpr int kDigitBits = 8;
constexpr int kRadix = 1 << kDigitBits;
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr uint32_t kScanSeg = kScanThreads * kScanItems;
constexpr uint32_t kBatch = 128;  // Sec. 4: batches of 128 points

// Keys per thread in flight in the write-out of a sort's last pass when it
// gathers the point records by index.
#ifndef PCR_GATHER_UNROLL
#define PCR_GATHER_UNROLL 8
#endif
constexpr int kGatherUnroll = PCR_GATHER_UNROLL;

static_assert(kRadix == kSortThreads, "one digit per thread in the sort kernels");
static_assert(kSortRounds % 4 == 0 && kShuffleRounds % 4 == 0, "keys per lane read as 16-byte vectors");

constexpr uint64_t align_up(uint64_t v) { return (v + 255) & ~uint64_t(255); }

constexpr uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

// Workspace layout; every region starts on a 256-byte boundary.
struct Layout {
  uint64_t pts_copy, keys0, keys1, vals0, vals1, counts, partials, bkeys0, bkeys1, bvals0, bvals1, misc, total;
};

constexpr uint64_t region(uint64_t& off, uint64_t bytes) {
  const uint64_t at = off;
  off += align_up(bytes > 0 ? bytes : 1);
  return at;
}

constexpr Layout layout(uint64_t n) {
  const uint64_t nb = ceil_div(n, kBatch);
  const uint64_t tiles = ceil_div(n > nb ? n : nb, kTileOf<kMinRounds>);  // the most any sort has
  const uint64_t count_words = kRadix * (tiles > 0 ? tiles : 1);
  Layout l{};
  uint64_t off = 0;
  l.pts_copy = region(off, 16 * n);
  l.keys0 = region(off, 4 * n);
  l.keys1 = region(off, 4 * n);
  l.vals0 = region(off, 4 * n);
  l.vals1 = region(off, 4 * n);
  l.counts = region(off, 4 * count_words);
  l.partials = region(off, 4 * ceil_div(count_words, kScanSeg));
  l.bkeys0 = region(off, 4 * nb);
  l.bkeys1 = region(off, 4 * nb);
  l.bvals0 = region(off, 4 * nb);
  l.bvals1 = region(off, 4 * nb);
  l.misc = region(off, 64);
  l.total = off;
  return l;
}

// --- bounds -------------------------------------------------------------------

// Order-preserving map from float to uint32 (NaN excluded by the caller).
__device__ __forceinline__ uint32_t float_order(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float order_float(uint32_t o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o);
}

__global__ void k_bounds_init(uint32_t* misc) {
  if (threadIdx.x < 3) {
    misc[threadIdx.x] = 0xFF800000u;     // order of +inf: identity for min
    misc[3 + threadIdx.x] = 0x007FFFFFu; // order of -inf: identity for max
  }
}

constexpr int kStreamUnroll = 4;
#ifndef PCR_MORTON_UNROLL
#define PCR_MORTON_UNROLL 8
#endif
constexpr int kMortonUnroll = PCR_MORTON_UNROLL;  // divides kSortRounds
static_assert(kSortRounds % kMortonUnroll == 0, "whole rounds of records per tile");

// Per axis min and max over non-NaN coordinates.  -0 is folded into +0 (the
// codes do not depend on the sign of a zero bound).  With `copy`, the records
// are also copied there (the source the sort's last pass moves them from),
// saving a pass.
__global__ void __launch_bounds__(256) k_bounds(const uint4* __restrict__ pts, uint32_t n, uint32_t* misc,
                                                uint4* __restrict__ copy) {
  uint32_t lo[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
  uint32_t hi[3] = {0u, 0u, 0u};
  // kStreamUnroll records per thread per step, all loads issued first
  const uint64_t step = gridDim.x * 256ull * kStreamUnroll;
  for (uint64_t i0 = blockIdx.x * 256ull * kStreamUnroll + threadIdx.x; i0 < n; i0 += step) {
    uint4 r[kStreamUnroll];
#pragma unroll
    for (int u = 0; u < kStreamUnroll; ++u) {
      const uint64_t i = i0 + 256ull * u;
      r[u] = i < n ? __ldcs(pts + i) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int u = 0; u < kStreamUnroll; ++u) {
      const uint64_t i = i0 + 256ull * u;
      if (i >= n) break;
      if (copy) __stcs(copy + i, r[u]);
      const float v[3] = {__uint_as_float(r[u].x), __uint_as_float(r[u].y), __uint_as_float(r[u].z)};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (v[a] == v[a]) {
          const uint32_t o = float_order(__fadd_rn(v[a], 0.0f));
          lo[a] = min(lo[a], o);
          hi[a] = max(hi[a], o);
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = __reduce_min_sync(kFullMask, lo[a]);
    hi[a] = __reduce_max_sync(kFullMask, hi[a]);
  }
  if (lane_id() == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (lo[a] != 0xFFFFFFFFu) atomicMin(misc + a, lo[a]);
      if (hi[a] != 0u) atomicMax(misc + 3 + a, hi[a]);
    }
  }
}

// --- codes --------------------------------------------------------------------

// Spread the low 10 bits of v so bit i lands on bit 3i.
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__device__ __forceinline__ uint32_t quantise(float v, float lo, float scale) {
  const float f = floorf(__fmul_rn(__fsub_rn(v, lo), scale));
  if (!(f >= 0.0f)) return 0u;
  if (f >= 1023.0f) return 1023u;
  return static_cast<uint32_t>(f);
}

// The kernels that make the keys also count the first sort pass's digits:
// one block per tile of kTile keys makes the tile's keys (thread t takes
// tile slots t, t + 256, ..., so loads and stores coalesce), keeps them in
// shared memory, and counts them as k_sort_hist does (with R keys per lane,
// lane l of warp w takes slots [32 R w + R l, + R) and adds each run of
// equal digits once), so the first pass's histogram costs no second read of
// the keys.
template <int ROUNDS>
struct alignas(16) TileKeys {
  uint32_t keys[kTileOf<ROUNDS>];  // read as 16-byte vectors by count_tile_digits
  uint32_t hist[kSortWarps][kRadix];
};

template <int ROUNDS>
__device__ __forceinline__ void count_tile_digits(TileKeys<ROUNDS>& sh, uint32_t valid, uint32_t* __restrict__ counts,
                                                  uint32_t tiles) {
  __syncthreads();  // the tile's keys are in place
  uint32_t* mine = sh.hist[threadIdx.x >> 5];
  const uint32_t first = (threadIdx.x >> 5) * (kTileOf<ROUNDS> / kSortWarps) + lane_id() * ROUNDS;
  uint32_t cur = 0, run = 0;
  if (first + ROUNDS <= valid) {
    const uint4* q = reinterpret_cast<const uint4*>(sh.keys + first);  // 16-byte aligned: 4 | ROUNDS
#pragma unroll
    for (int k = 0; k < ROUNDS / 4; ++k) {
      const uint4 v = q[k];
      const uint32_t d[4] = {v.x & (kRadix - 1), v.y & (kRadix - 1), v.z & (kRadix - 1), v.w & (kRadix - 1)};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (d[e] == cur) {
          ++run;
        } else {
          if (run) atomicAdd(&mine[cur], run);
          cur = d[e];
          run = 1;
        }
      }
    }
  } else {
    for (uint32_t j = first; j < valid && j < first + ROUNDS; ++j) {
      const uint32_t d = sh.keys[j] & (kRadix - 1);
      if (d == cur) {
        ++run;
      } else {
        if (run) atomicAdd(&mine[cur], run);
        cur = d;
        run = 1;
      }
    }
  }
  if (run) atomicAdd(&mine[cur], run);
  __syncthreads();
  uint32_t c = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) c += sh.hist[w][threadIdx.x];
  counts[static_cast<uint64_t>(threadIdx.x) * tiles + blockIdx.x] = c;
}

template <int ROUNDS>
__device__ __forceinline__ void zero_tile_hist(TileKeys<ROUNDS>& sh) {
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) sh.hist[w][threadIdx.x] = 0;
}


// Sec. 5: Morton code over the cube with the bounds' minimum corner and the
// largest extent as side, 10 levels.
__global__ void __launch_bounds__(kSortThreads) k_morton(const uint4* __restrict__ pts, uint32_t n,
                                                         const uint32_t* __restrict__ misc,
                                                         uint32_t* __restrict__ keys, uint32_t* __restrict__ counts,
                                                         uint32_t tiles) {
  __shared__ TileKeys<kSortRounds> sh;
  zero_tile_hist(sh);
  const float lo[3] = {order_float(misc[0]), order_float(misc[1]), order_float(misc[2])};
  const float hi[3] = {order_float(misc[3]), order_float(misc[4]), order_float(misc[5])};
  float ext = __fsub_rn(hi[0], lo[0]);
  const float ey = __fsub_rn(hi[1], lo[1]);
  const float ez = __fsub_rn(hi[2], lo[2]);
  if (ey > ext) ext = ey;
  if (ez > ext) ext = ez;
  const bool degenerate = !(ext > 0.0f) || !(ext < __int_as_float(kInfBits));
  const float scale = degenerate ? 0.0f : __fdiv_rn(1024.0f, ext);
  const uint64_t tile_base = static_cast<uint64_t>(blockIdx.x) * kTile;
  const uint32_t valid = static_cast<uint32_t>(n - tile_base < kTile ? n - tile_base : kTile);
  // kMortonUnroll records per thread in flight at a time
  for (uint32_t j0 = threadIdx.x; j0 < valid; j0 += kSortThreads * kMortonUnroll) {
    uint4 r[kMortonUnroll];
#pragma unroll
    for (int u = 0; u < kMortonUnroll; ++u) {
      const uint32_t j = j0 + kSortThreads * u;
      r[u] = (!degenerate && j < valid) ? __ldcs(pts + tile_base + j) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int u = 0; u < kMortonUnroll; ++u) {
      const uint32_t j = j0 + kSortThreads * u;
      if (j >= valid) break;
      uint32_t code = 0;
      if (!degenerate) {
        code = (spread3(quantise(__uint_as_float(r[u].x), lo[0], scale)) << 2) |
               (spread3(quantise(__uint_as_float(r[u].y), lo[1], scale)) << 1) |
               spread3(quantise(__uint_as_float(r[u].z), lo[2], scale));
      }
      keys[tile_base + j] = code;
      sh.keys[j] = code;
    }
  }
  count_tile_digits(sh, valid, counts, tiles);
}

// Spread the low 21 bits of v so bit i lands on bit 3i.
__device__ __forceinline__ uint64_t spread3_21(uint32_t x) {
  uint64_t v = x & 0x1FFFFFu;
  v = (v | (v << 32)) & 0x001F00000000FFFFull;
  v = (v | (v << 16)) & 0x001F0000FF0000FFull;
  v = (v | (v << 8)) & 0x100F00F00F00F00Full;
  v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

__device__ __forceinline__ uint32_t quantise21(float v, float lo, float scale) {
  const float f = floorf(__fmul_rn(__fsub_rn(v, lo), scale));
  if (!(f >= 0.0f)) return 0u;
  if (f >= 2097151.0f) return 2097151u;
  return static_cast<uint32_t>(f);
}

// Sec. 5 with the paper's 21 levels: the same cube, 2^21 cells per axis.
// Writes the code's low 32 bits to keys_lo and its high 31 bits to hi.
__global__ void __launch_bounds__(kSortThreads) k_morton63(const uint4* __restrict__ pts, uint32_t n,
                                                           const uint32_t* __restrict__ misc,
                                                           uint32_t* __restrict__ keys_lo, uint32_t* __restrict__ hi,
                                                           uint32_t* __restrict__ counts, uint32_t tiles) {
  __shared__ TileKeys<kSortRounds> sh;
  zero_tile_hist(sh);
  const float lo[3] = {order_float(misc[0]), order_float(misc[1]), order_float(misc[2])};
  const float top[3] = {order_float(misc[3]), order_float(misc[4]), order_float(misc[5])};
  float ext = __fsub_rn(top[0], lo[0]);
  const float ey = __fsub_rn(top[1], lo[1]);
  const float ez = __fsub_rn(top[2], lo[2]);
  if (ey > ext) ext = ey;
  if (ez > ext) ext = ez;
  const bool degenerate = !(ext > 0.0f) || !(ext < __int_as_float(kInfBits));
  const float scale = degenerate ? 0.0f : __fdiv_rn(2097152.0f, ext);
  const uint64_t tile_base = static_cast<uint64_t>(blockIdx.x) * kTile;
  const uint32_t valid = static_cast<uint32_t>(n - tile_base < kTile ? n - tile_base : kTile);
  for (uint32_t j = threadIdx.x; j < valid; j += kSortThreads) {
    uint64_t code = 0;
    if (!degenerate) {
      const uint4 r = __ldcs(pts + tile_base + j);
      code = (spread3_21(quantise21(__uint_as_float(r.x), lo[0], scale)) << 2) |
             (spread3_21(quantise21(__uint_as_float(r.y), lo[1], scale)) << 1) |
             spread3_21(quantise21(__uint_as_float(r.z), lo[2], scale));
    }
    keys_lo[tile_base + j] = static_cast<uint32_t>(code);
    hi[tile_base + j] = static_cast<uint32_t>(code >> 32);
    sh.keys[j] = static_cast<uint32_t>(code);
  }
  count_tile_digits(sh, valid, counts, tiles);
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): output k of the generator
// seeded with `seed` mixes the state seed + (k + 1) * 0x9E3779B97F4A7C15.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Keys for the random orders: the high half of SplitMix64 output i, with the
// first sort pass's digit counts.
template <int ROUNDS>
__global__ void __launch_bounds__(kSortThreads) k_random_keys(uint32_t count, uint64_t seed,
                                                              uint32_t* __restrict__ keys,
                                                              uint32_t* __restrict__ counts, uint32_t tiles) {
  __shared__ TileKeys<ROUNDS> sh;
  zero_tile_hist(sh);
  constexpr uint32_t kT = kTileOf<ROUNDS>;
  const uint64_t tile_base = static_cast<uint64_t>(blockIdx.x) * kT;
  const uint32_t valid = static_cast<uint32_t>(count - tile_base < kT ? count - tile_base : kT);
  for (uint32_t j = threadIdx.x; j < valid; j += kSortThreads) {
    const uint32_t key = static_cast<uint32_t>(splitmix64(seed, tile_base + j) >> 32);
    keys[tile_base + j] = key;
    sh.keys[j] = key;
  }
  count_tile_digits(sh, valid, counts, tiles);
}

// --- radix sort ---------------------------------------------------------------

// Lanes of the warp whose 8-bit digit equals this lane's, among the lanes
// in `valid`.  When the warp's digits form few runs (coherent keys: a
// Morton order's high digits), one match.any finds them cheaply; otherwise
// one ballot per digit bit does, at a cost that does not depend on how many
// distinct digits the warp holds (match.any grows with that number).
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, uint32_t valid) {
  const uint32_t prev = __shfl_up_sync(kFullMask, d, 1);
  const uint32_t runs = __popc(__ballot_sync(kFullMask, lane_id() == 0 || prev != d));
  if (runs <= 6) return __match_any_sync(kFullMask, d) & valid;
  uint32_t peers = valid;
#pragma unroll
  for (int b = 0; b < kDigitBits; ++b) {
    const uint32_t bit = (d >> b) & 1u;
    const uint32_t set = __ballot_sync(kFullMask, bit);
    peers &= bit ? set : ~set;
  }
  return peers;
}

// Per tile, the count of each digit.  With R keys per lane, lane l of each
// warp counts keys [R l, R l + R) of the warp's 32 R (16-byte loads) and
// adds a run of equal digits to its warp's counters once, when the digit
// changes.
// Coherent orders (and the passes after the first, whose input is sorted on
// the lower digits) have long runs, which one add per key would turn into
// many same-address shared-memory atomics.  The eight warps' counters are
// summed at the end.
template <int ROUNDS>
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint32_t* __restrict__ keys, uint32_t n, int shift,
                                                            uint32_t* __restrict__ counts, uint32_t tiles) {
  __shared__ uint32_t hist[kSortWarps][kRadix];
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) hist[w][threadIdx.x] = 0;
  __syncthreads();
  uint32_t* mine = hist[threadIdx.x >> 5];
  const uint64_t first = static_cast<uint64_t>(blockIdx.x) * kTileOf<ROUNDS> +
                         (threadIdx.x >> 5) * (kTileOf<ROUNDS> / kSortWarps) + lane_id() * ROUNDS;
  uint32_t cur = 0, run = 0;
  auto count = [&](uint32_t key) {
    const uint32_t d = (key >> shift) & (kRadix - 1);
    if (d == cur) {
      ++run;
    } else {
      if (run) atomicAdd(&mine[cur], run);
      cur = d;
      run = 1;
    }
  };
  if (first + ROUNDS <= n) {
    const uint4* q = reinterpret_cast<const uint4*>(keys + first);  // 16-byte aligned: 4 | ROUNDS
    uint4 v[ROUNDS / 4];
#pragma unroll
    for (int k = 0; k < ROUNDS / 4; ++k) v[k] = __ldg(q + k);
#pragma unroll
    for (int k = 0; k < ROUNDS / 4; ++k) {
      count(v[k].x);
      count(v[k].y);
      count(v[k].z);
      count(v[k].w);
    }
  } else {
    for (uint64_t i = first; i < n && i < first + ROUNDS; ++i) count(__ldg(keys + i));
  }
  if (run) atomicAdd(&mine[cur], run);
  __syncthreads();
  uint32_t c = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) c += hist[w][threadIdx.x];
  counts[static_cast<uint64_t>(threadIdx.x) * tiles + blockIdx.x] = c;
}

template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t& total);


// Dynamic shared memory of k_sort_scatter: the tile's keys as loaded, each
// output slot's input slot, the per-warp first slot of each digit, and per
// digit the output position minus the tile slot of its first key.  45 KB for
// 24 keys per lane, 38 KB for 20: four blocks per SM either way.
template <int ROUNDS>
constexpr size_t scatter_smem() {
  return sizeof(uint32_t) * kTileOf<ROUNDS> + sizeof(uint16_t) * kTileOf<ROUNDS> +
         sizeof(uint32_t) * (kSortWarps * kRadix + kRadix);
}

// 16-byte asynchronous copy global -> shared (cp.async, completes on
// cp.async.wait_all); `bytes` < 16 reads only that many and zero-fills.
__device__ __forceinline__ void copy16_async(void* smem_dst, const void* gmem_src, uint32_t bytes) {
  const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(gmem_src), "r"(bytes) : "memory");
}

// The last pass of a sort may move the point records itself: the record at
// each key's value (an index into `src`) goes straight to the key's final
// position, so the permutation makes no round trip through memory and no
// gather pass follows.  With `rank`, final positions are those of the
// 128-point batch order (Sec. 4): sorted position g lies in batch g / 128,
// which goes to batch slot rank[g / 128], and slots after the short last
// batch start (128 - its size) earlier.
struct FinalGather {
  const uint4* src = nullptr;      // records by input index; null: no gather
  uint4* dst = nullptr;            // records by final position
  uint32_t* perm_out = nullptr;    // optional: final position -> input index
  const uint32_t* rank = nullptr;  // optional: batch -> its slot in the batch order
  uint32_t nb = 0;                 // batches (with rank)
};

// `kout` may be null: the last pass of a sort writes no keys (nothing reads
// them).  `cin`/`cout` (may be null): a second 32-bit value carried with each
// key (the high words of 63-bit codes while their low words are sorted).
// `vout` may be null when no value is carried; a null `vin` with a `vout`
// carries each key's input index (the first pass of a sort whose values start
// as the identity, so they are never written out and read back).  With REC,
// the 16-byte point record `rin[i]` moves with its key to `rout` (the random
// order sorts the records themselves: every pass reads them in tile order and
// writes them in digit runs, instead of one random gather at the end).  With
// `fin.src` the records move as FinalGather says, and `vout` is not written.
template <bool REC, int ROUNDS>
__global__ void __launch_bounds__(kSortThreads, 4) k_sort_scatter(const uint32_t* __restrict__ kin,
                                                                  const uint32_t* __restrict__ vin,
                                                                  uint32_t* __restrict__ kout,
                                                                  uint32_t* __restrict__ vout, uint32_t n, int shift,
                                                                  const uint32_t* __restrict__ offsets,
                                                                  uint32_t tiles, const uint32_t* __restrict__ cin,
                                                                  uint32_t* __restrict__ cout,
                                                                  const uint4* __restrict__ rin,
                                                                  uint4* __restrict__ rout, FinalGather fin) {
  constexpr uint32_t kT = kTileOf<ROUNDS>;  // keys in a tile
  constexpr uint32_t kKeysPerWarp = kT / kSortWarps;
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* s_kin = smem;                                         // [kT] the tile's keys
  uint32_t* wbase = s_kin + kT;                                   // [kSortWarps][kRadix]
  uint32_t* delta = wbase + kSortWarps * kRadix;                  // [kRadix]
  uint16_t* s_src = reinterpret_cast<uint16_t*>(delta + kRadix);  // [kT]
  const uint32_t t = threadIdx.x;
  const uint32_t lane = lane_id();
  const uint32_t warp = t >> 5;
  const uint64_t tile_base = static_cast<uint64_t>(blockIdx.x) * kT;
  const uint32_t valid = static_cast<uint32_t>(n - tile_base < kT ? n - tile_base : kT);
  for (uint32_t c = t; c * 4 < valid; c += kSortThreads) {
    const uint32_t left = valid - 4 * c;
    copy16_async(s_kin + 4 * c, kin + tile_base + 4ull * c, left >= 4 ? 16u : 4 * left);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) wbase[w * kRadix + t] = 0;
  const uint32_t global_start = offsets[static_cast<uint64_t>(t) * tiles + blockIdx.x];
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  // this warp's 768 consecutive keys; pass 1 counts their digits, and each
  // key keeps its rank among the round's lanes with its digit, that group's
  // size and the digit (rank | size << 8 | digit << 16, bit 31 set for a key
  // inside the cloud)
  const uint32_t wfirst = warp * kKeysPerWarp;
  uint32_t* mine = wbase + warp * kRadix;
  const uint32_t below = (1u << lane) - 1u;
  uint32_t info[ROUNDS];
  // a full tile (every tile but a cloud's last) needs no test of which keys
  // lie inside the cloud
  auto rank_keys = [&](auto full) {
    constexpr bool kFull = decltype(full)::value;
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
      const uint32_t j = wfirst + r * 32 + lane;
      const bool ok = kFull || j < valid;
      const uint32_t d = ok ? (s_kin[j] >> shift) & (kRadix - 1) : 0u;
      const uint32_t peers = digit_peers(d, kFull ? kFullMask : __ballot_sync(kFullMask, ok));
      const uint32_t rank = __popc(peers & below);
      info[r] = ok ? (rank | (static_cast<uint32_t>(__popc(peers)) << 8) | (d << 16) | 0x80000000u) : 0u;
      if (ok && rank == 0) mine[d] += __popc(peers);
      __syncwarp();
    }
  };
  if (valid == kT) rank_keys(std::true_type{});
  else rank_keys(std::false_type{});
  __syncthreads();
  // digit t: first slot of each warp's keys within the digit, then the
  // digit's first slot within the tile
  uint32_t run = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {
    const uint32_t c = wbase[w * kRadix + t];
    wbase[w * kRadix + t] = run;
    run += c;
  }
  uint32_t total;
  const uint32_t start = block_exclusive_scan<kSortThreads>(run, total);
  delta[t] = global_start - start;  // modulo 2^32: output position = delta + tile slot
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) wbase[w * kRadix + t] += start;
  __syncthreads();
  // pass 2: each key's slot in the tile's digit order, in index order
  auto place_keys = [&](auto full) {
    constexpr bool kFull = decltype(full)::value;
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
      const uint32_t v = info[r];
      const bool ok = kFull || (v >> 31) != 0u;
      const uint32_t d = (v >> 16) & (kRadix - 1);
      const uint32_t rank = v & 0xFFu;
      const uint32_t at = ok ? mine[d] : 0u;
      __syncwarp();
      if (ok && debug_in_range(at + rank, kT)) {
        s_src[at + rank] = static_cast<uint16_t>(wfirst + r * 32 + lane);
        if (rank == 0) mine[d] = at + ((v >> 8) & 0xFFu);
      }
      __syncwarp();
    }
  };
  if (valid == kT) place_keys(std::true_type{});
  else place_keys(std::false_type{});
  __syncthreads();
  // the tile in digit order: consecutive slots of a digit go to consecutive
  // output positions; values are gathered from the tile's window.  One
  // loop per combination of what moves with the keys, chosen once, so each
  // unrolled loop carries no per-key test.
  auto write_out = [&](auto values, auto carried, auto keys, auto gather, auto perm) {
    constexpr int kValues = decltype(values)::value;  // 0 none, 1 loaded, 2 the key's index
    constexpr bool kCarried = decltype(carried)::value;
    constexpr bool kKeys = decltype(keys)::value;
    constexpr int kGather = decltype(gather)::value;  // 0 none, 1 to sorted position, 2 to batch order
    constexpr bool kPerm = decltype(perm)::value;
    uint32_t t_last = 0, short_by = 0;
    if constexpr (kGather == 2) {
      t_last = __ldg(fin.rank + (fin.nb - 1));
      short_by = fin.nb * kBatch - n;
    }
    auto one = [&](uint32_t l) {
      const uint32_t src = s_src[l];
      const uint32_t key = s_kin[src];
      const uint32_t d = (key >> shift) & (kRadix - 1);
      const uint32_t g = delta[d] + l;
      if (!debug_in_range(g, n)) return;
      if constexpr (kKeys) kout[g] = key;
      uint32_t v = 0;
      if constexpr (kValues == 1) v = __ldg(vin + tile_base + src);
      if constexpr (kValues == 2) v = static_cast<uint32_t>(tile_base + src);
      if constexpr (kGather == 0) {
        if constexpr (kValues != 0) vout[g] = v;
      } else {
        uint32_t at = g;
        if constexpr (kGather == 2) {
          const uint32_t slot = __ldg(fin.rank + g / kBatch);
          at = slot * kBatch + g % kBatch - (slot > t_last ? short_by : 0u);
        }
        if (!debug_in_range(v, n) || !debug_in_range(at, n)) return;
        __stcs(fin.dst + at, __ldg(fin.src + v));
        if constexpr (kPerm) fin.perm_out[at] = v;
      }
      if constexpr (kCarried) cout[g] = __ldg(cin + tile_base + src);
      if constexpr (REC) __stcs(rout + g, __ldg(rin + tile_base + src));
    };
    // records carried: one key per iteration (unrolled 2, 3, 4 or 8 times the
    // 800M shuffle took 36.2, 35.9, 38.1 and 39.2 ms against 35.4); records
    // gathered by index: kGatherUnroll; keys and 4-byte values: eight
    if constexpr (REC) {
#pragma unroll 1
      for (uint32_t l = t; l < total; l += kSortThreads) one(l);
    } else if constexpr (kGather != 0) {
#pragma unroll kGatherUnroll
      for (uint32_t l = t; l < total; l += kSortThreads) one(l);
    } else {
#pragma unroll 8
      for (uint32_t l = t; l < total; l += kSortThreads) one(l);
    }
  };
  using C0 = std::integral_constant<int, 0>;
  using C1 = std::integral_constant<int, 1>;
  using C2 = std::integral_constant<int, 2>;
  using Yes = std::true_type;
  using No = std::false_type;
  if constexpr (!REC) {
    if (fin.src) {
      auto go = [&](auto values) {
        if (fin.rank) {
          if (fin.perm_out) write_out(values, No{}, No{}, C2{}, Yes{});
          else write_out(values, No{}, No{}, C2{}, No{});
        } else {
          if (fin.perm_out) write_out(values, No{}, No{}, C1{}, Yes{});
          else write_out(values, No{}, No{}, C1{}, No{});
        }
      };
      if (vin) go(C1{});
      else go(C2{});
      return;
    }
  }
  auto go = [&](auto values) {
    if constexpr (REC) {
      if (kout) write_out(values, No{}, Yes{}, C0{}, No{});
      else write_out(values, No{}, No{}, C0{}, No{});
    } else {
      if (kout) {
        if (cout) write_out(values, Yes{}, Yes{}, C0{}, No{});
        else write_out(values, No{}, Yes{}, C0{}, No{});
      } else {
        if (cout) write_out(values, Yes{}, No{}, C0{}, No{});
        else write_out(values, No{}, No{}, C0{}, No{});
      }
    }
  };
  if (!vout) go(C0{});
  else if (vin) go(C1{});
  else go(C2{});
}

// --- exclusive scan (in place) ----------------------------------------------------

template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t& total) {
  __shared__ uint32_t warp_sums[NT / 32];
  const uint32_t lane = lane_id();
  const uint32_t warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFullMask, x, o);
    if (lane >= static_cast<uint32_t>(o)) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < NT / 32 ? warp_sums[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFullMask, s, o);
      if (lane >= static_cast<uint32_t>(o)) s += y;
    }
    if (lane < NT / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  total = warp_sums[NT / 32 - 1];
  const uint32_t prefix = warp ? warp_sums[warp - 1] : 0u;
  return prefix + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ a, uint64_t len,
                                                              uint32_t* __restrict__ partials) {
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kScanSeg + threadIdx.x;
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const uint64_t i = base + static_cast<uint64_t>(j) * kScanThreads;
    if (i < len) s += a[i];
  }
  s = __reduce_add_sync(kFullMask, s);
  __shared__ uint32_t w[kScanThreads / 32];
  if (lane_id() == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int k = 0; k < kScanThreads / 32; ++k) t += w[k];
    partials[blockIdx.x] = t;
  }
}

// One block of 1024 threads; thread t scans a contiguous run of partials.
__global__ void __launch_bounds__(1024) k_scan_partials(uint32_t* __restrict__ partials, uint32_t count) {
  const uint32_t per = (count + 1023) / 1024;
  const uint64_t first = static_cast<uint64_t>(threadIdx.x) * per;
  uint32_t local = 0;
  for (uint32_t j = 0; j < per; ++j)
    if (first + j < count) local += partials[first + j];
  uint32_t total;
  uint32_t run = block_exclusive_scan<1024>(local, total);
  for (uint32_t j = 0; j < per; ++j) {
    if (first + j < count) {
      const uint32_t v = partials[first + j];
      partials[first + j] = run;
      run += v;
    }
  }
}

// Thread t scans the 16 consecutive counts [16 t, 16 t + 16) of its block's
// segment, read and written as four 16-byte vectors (segments start on
// 16-KB boundaries of the count array), so no shared-memory staging is
// needed.
__global__ void __launch_bounds__(kScanThreads) k_scan_down(uint32_t* __restrict__ a, uint64_t len,
                                                            const uint32_t* __restrict__ partials) {
  static_assert(kScanItems == 16, "four 16-byte vectors per thread");
  const uint64_t first = static_cast<uint64_t>(blockIdx.x) * kScanSeg + static_cast<uint64_t>(threadIdx.x) * kScanItems;
  uint32_t mine[kScanItems];
  const bool whole = first + kScanItems <= len;
  if (whole) {
    const uint4* q = reinterpret_cast<const uint4*>(a + first);
#pragma unroll
    for (int k = 0; k < kScanItems / 4; ++k) {
      const uint4 v = q[k];
      mine[4 * k] = v.x;
      mine[4 * k + 1] = v.y;
      mine[4 * k + 2] = v.z;
      mine[4 * k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) mine[j] = first + j < len ? a[first + j] : 0u;
  }
  uint32_t sum = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) sum += mine[j];
  uint32_t total;
  uint32_t run = block_exclusive_scan<kScanThreads>(sum, total) + partials[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const uint32_t v = mine[j];
    mine[j] = run;
    run += v;
  }
  if (whole) {
    uint4* q = reinterpret_cast<uint4*>(a + first);
#pragma unroll
    for (int k = 0; k < kScanItems / 4; ++k)
      q[k] = make_uint4(mine[4 * k], mine[4 * k + 1], mine[4 * k + 2], mine[4 * k + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
      if (first + j < len) a[first + j] = mine[j];
  }
}

cudaError_t exclusive_scan(uint32_t* a, uint64_t len, uint32_t* partials, cudaStream_t s) {
  const uint64_t blocks = ceil_div(len, kScanSeg);
  k_scan_reduce<<<static_cast<unsigned>(blocks), kScanThreads, 0, s>>>(a, len, partials);
  k_scan_partials<<<1, 1024, 0, s>>>(partials, static_cast<uint32_t>(blocks));
  k_scan_down<<<static_cast<unsigned>(blocks), kScanThreads, 0, s>>>(a, len, partials);
  return cudaGetLastError();
}

// Stable sort of count (key, value) pairs on the low key_bits bits.  The
// result ends in buffer index `out` (0 or 1): the values, and the carried
// words; the last pass writes no keys.  With `carry` (may be null), a second
// value per key moves with it through its own two buffers, and with
// `carry_last` (may be null) the last pass writes the carried words there
// instead.  With `recs` (may be null), a 16-byte record moves with each key.
// vals may hold null buffers when no value is needed.  With `index_values`
// the values start as each key's index: the first pass makes them, and
// vals[0] is never read.  With `first_counted` the kernel that made the keys
// has already written the first pass's digit counts (k_morton, k_morton63,
// k_random_keys).  With `fin` (may be null) the last pass moves the records
// as FinalGather says, instead of writing the values.
template <int ROUNDS>
cudaError_t radix_sort(uint32_t* keys[2], uint32_t* vals[2], uint32_t count, int key_bits, uint32_t* counts,
                       uint32_t* partials, cudaStream_t s, int& out, bool index_values, bool first_counted,
                       uint32_t* const* carry = nullptr, uint32_t* carry_last = nullptr,
                       uint4* const* recs = nullptr, const FinalGather* fin = nullptr) {
  out = 0;
  if (count == 0) return cudaSuccess;
  constexpr size_t kSmem = scatter_smem<ROUNDS>();
  const uint32_t tiles = static_cast<uint32_t>(ceil_div(count, kTileOf<ROUNDS>));
  cudaError_t e = cudaFuncSetAttribute(recs ? k_sort_scatter<true, ROUNDS> : k_sort_scatter<false, ROUNDS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kSmem));
  if (e != cudaSuccess) return e;
  for (int shift = 0; shift < key_bits; shift += kDigitBits) {
    const bool last = shift + kDigitBits >= key_bits;
    if (!(first_counted && shift == 0)) k_sort_hist<ROUNDS><<<tiles, kSortThreads, 0, s>>>(keys[out], count, shift, counts, tiles);
    e = exclusive_scan(counts, static_cast<uint64_t>(kRadix) * tiles, partials, s);
    if (e != cudaSuccess) return e;
    const uint32_t* vin = (index_values && shift == 0) ? nullptr : vals[out];
    uint32_t* kout = last ? nullptr : keys[out ^ 1];
    const FinalGather f = (last && fin) ? *fin : FinalGather{};
    if (recs)
      k_sort_scatter<true, ROUNDS><<<tiles, kSortThreads, kSmem, s>>>(
          keys[out], vin, kout, vals[out ^ 1], count, shift, counts, tiles, nullptr, nullptr, recs[out],
          recs[out ^ 1], f);
    else
      k_sort_scatter<false, ROUNDS><<<tiles, kSortThreads, kSmem, s>>>(
          keys[out], vin, kout, vals[out ^ 1], count, shift, counts, tiles, carry ? carry[out] : nullptr,
          carry ? (last && carry_last ? carry_last : carry[out ^ 1]) : nullptr, nullptr, nullptr, f);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    out ^= 1;
  }
  return cudaSuccess;
}

// --- shuffled Morton: batch slots; record copy -------------------------------------

// Slot of each batch in the sorted batch order: rank[order[t]] = t.
__global__ void k_batch_rank(const uint32_t* __restrict__ order, uint32_t nb, uint32_t* __restrict__ rank) {
  for (uint64_t t = blockIdx.x * 256ull + threadIdx.x; t < nb; t += gridDim.x * 256ull) {
    const uint32_t b = order[t];
    if (debug_in_range(b, nb)) rank[b] = static_cast<uint32_t>(t);
  }
}

__global__ void __launch_bounds__(256) k_copy16(const uint4* __restrict__ src, uint4* __restrict__ dst, uint32_t n) {
  for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < n; i += gridDim.x * 256ull) dst[i] = __ldcs(src + i);
}

unsigned stream_grid(uint64_t count, const Device& d) {
  const uint64_t need = ceil_div(count, 256);
  const uint64_t cap = static_cast<uint64_t>(d.num_sms) * 8;
  return static_cast<unsigned>(need < cap ? (need > 0 ? need : 1) : cap);
}

}  // namespace

// Scratch for the allocation-free reorder: one workspace sized for the
// largest accepted cloud, part of the module's device memory.
constexpr uint64_t kNoallocScratchBytes = layout(PCR_REORDER_NOALLOC_MAX_POINTS).total;
static __device__ __align__(256) unsigned char g_reorder_scratch[kNoallocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_reorder_scratch on `device`, looked up once per device
// with that device current (host code cannot use the symbol itself).  A new
// context on the device (pcr_create) drops the cached address, so a process
// that reset the device and created a new context looks it up again.
cudaError_t noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (g_scratch_addr[device] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_reorder_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

}  // namespace

void forget_noalloc_scratch(int device) {
  if (device < 0 || device >= kMaxDevices) return;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  g_scratch_addr[device] = nullptr;
}

uint64_t reorder_workspace_bytes(uint64_t n) { return layout(n).total; }

cudaError_t launch_reorder(uint4* pts, uint32_t n, uint64_t seed, int mode, void* workspace, uint32_t* perm_out,
                           cudaStream_t s, const Device& d) {
  if (n == 0) return cudaSuccess;
  const Layout l = layout(n);
  char* ws = static_cast<char*>(workspace);
  uint4* copy = reinterpret_cast<uint4*>(ws + l.pts_copy);
  uint32_t* keys[2] = {reinterpret_cast<uint32_t*>(ws + l.keys0), reinterpret_cast<uint32_t*>(ws + l.keys1)};
  uint32_t* vals[2] = {reinterpret_cast<uint32_t*>(ws + l.vals0), reinterpret_cast<uint32_t*>(ws + l.vals1)};
  uint32_t* counts = reinterpret_cast<uint32_t*>(ws + l.counts);
  uint32_t* partials = reinterpret_cast<uint32_t*>(ws + l.partials);
  uint32_t* misc = reinterpret_cast<uint32_t*>(ws + l.misc);
  const unsigned grid = stream_grid(n, d);
  const uint32_t tiles = static_cast<uint32_t>(ceil_div(n, kTile));  // the sort's tiles
  cudaError_t e = cudaSuccess;
  int out = 0;
  if (mode == PCR_ORDER_SHUFFLE) {
    // the records themselves are sorted by their random keys (4 passes, an
    // even number: they end back in the caller's buffer); indices ride along
    // only when the permutation is asked for, with the caller's buffer as
    // the value buffer the last pass writes
    const uint32_t stiles = static_cast<uint32_t>(ceil_div(n, kTileOf<kShuffleRounds>));
    k_random_keys<kShuffleRounds><<<stiles, kSortThreads, 0, s>>>(n, seed, keys[0], counts, stiles);
    uint32_t* ivals[2] = {perm_out, perm_out ? vals[1] : nullptr};
    uint4* recs[2] = {pts, copy};
    e = radix_sort<kShuffleRounds>(keys, ivals, n, 32, counts, partials, s, out, true, true, nullptr, nullptr, recs);
    if (e != cudaSuccess) return e;
    if (out != 0) return cudaErrorUnknown;  // 32-bit keys take 4 passes: the values end in ivals[0]
    return cudaSuccess;
  }
  // The sort's last pass moves the records from their copy to their final
  // positions: the sorted positions, or with the batch shuffle, the slots of
  // the batches' random order, which is sorted first.
  FinalGather fin;
  fin.src = copy;
  fin.dst = pts;
  fin.perm_out = perm_out;
  if (mode == PCR_ORDER_MORTON_SHUFFLE128 || mode == PCR_ORDER_MORTON63_SHUFFLE128) {
    const uint32_t nb = static_cast<uint32_t>(ceil_div(n, kBatch));
    uint32_t* bkeys[2] = {reinterpret_cast<uint32_t*>(ws + l.bkeys0), reinterpret_cast<uint32_t*>(ws + l.bkeys1)};
    uint32_t* bvals[2] = {reinterpret_cast<uint32_t*>(ws + l.bvals0), reinterpret_cast<uint32_t*>(ws + l.bvals1)};
    const uint32_t btiles = static_cast<uint32_t>(ceil_div(nb, kTile));
    k_random_keys<kSortRounds><<<btiles, kSortThreads, 0, s>>>(nb, seed, bkeys[0], counts, btiles);
    int bout = 0;
    e = radix_sort<kSortRounds>(bkeys, bvals, nb, 32, counts, partials, s, bout, true, true);
    if (e != cudaSuccess) return e;
    k_batch_rank<<<stream_grid(nb, d), 256, 0, s>>>(bvals[bout], nb, bkeys[0]);
    fin.rank = bkeys[0];
    fin.nb = nb;
  }
  k_bounds_init<<<1, 32, 0, s>>>(misc);
  if (mode == PCR_ORDER_MORTON || mode == PCR_ORDER_MORTON_SHUFFLE128) {
    k_bounds<<<grid, 256, 0, s>>>(pts, n, misc, copy);
    k_morton<<<tiles, kSortThreads, 0, s>>>(pts, n, misc, keys[0], counts, tiles);
    e = radix_sort<kSortRounds>(keys, vals, n, 30, counts, partials, s, out, true, true, nullptr, nullptr, nullptr,
                                &fin);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  // 63-bit code: the high halves ride along with their keys while the low
  // halves are sorted, in two buffers in the record-copy region; the last
  // pass leaves them in keys[0] (the low halves are no longer needed), which
  // frees the region for the record copy.  Then the high halves are sorted,
  // and that sort's last pass moves the records.
  uint32_t* hi[2] = {reinterpret_cast<uint32_t*>(ws + l.pts_copy),
                     reinterpret_cast<uint32_t*>(ws + l.pts_copy) + align_up(4ull * n) / 4};
  k_bounds<<<grid, 256, 0, s>>>(pts, n, misc, nullptr);
  k_morton63<<<tiles, kSortThreads, 0, s>>>(pts, n, misc, keys[0], hi[0], counts, tiles);
  int a = 0;
  e = radix_sort<kSortRounds>(keys, vals, n, 32, counts, partials, s, a, true, true, hi, keys[0]);
  if (e != cudaSuccess) return e;
  if (a != 0) return cudaErrorUnknown;  // 4 passes: the values are in vals[0]
  k_copy16<<<grid, 256, 0, s>>>(pts, copy, n);
  e = radix_sort<kSortRounds>(keys, vals, n, 31, counts, partials, s, out, false, false, nullptr, nullptr, nullptr,
                              &fin);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t read_and_clear_reorder_error_word(uint32_t* out, cudaStream_t s) {
  *out = 0;
#ifdef PCR_DEBUG
  const uint32_t zero = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_reorder_error_word, sizeof(uint32_t), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_reorder_error_word, &zero, sizeof(uint32_t), 0,
                                                    cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
#else
  (void)s;
  return cudaSuccess;
#endif
}

cudaError_t launch_reorder_noalloc(uint4* pts, uint32_t n, uint64_t seed, int mode, uint32_t* perm_out,
                                   cudaStream_t s, const Device& d) {
  if (n > PCR_REORDER_NOALLOC_MAX_POINTS) return cudaErrorInvalidValue;
  void* scratch = nullptr;
  const cudaError_t e = noalloc_scratch(d.id, &scratch);
  if (e != cudaSuccess) return e;
  return launch_reorder(pts, n, seed, mode, scratch, perm_out, s, d);
}

}  // namespace pcr
