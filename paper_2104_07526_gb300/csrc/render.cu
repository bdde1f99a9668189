// Render, high-quality and resolve kernels (Sec. 3 of Schuetz, Kerbl, Wimmer,
// "Rendering Point Clouds with Compute Shaders and Vertex Order
// Optimization", EGSR 2021).
//
// Geometry passes stream the 16-byte point records once each.  A warp takes a
// chunk of 32*U consecutive points (U per lane, lane-interleaved so every
// load instruction covers 512 contiguous bytes); a persistent grid of
// (SM count x resident blocks) walks the chunks in order, so the GPU works on
// a moving window of the buffer, as a vertex-order study needs.
#include <cstdint>
#include <type_traits>

#include "../../include/pcr.h"
#include "common.cuh"
#include "launch.h"

namespace pcr {

namespace {

__device__ uint32_t g_error_word;

#ifndef PCR_GEOMETRY_UNROLL
#define PCR_GEOMETRY_UNROLL 4
#endif
#ifndef PCR_GEOMETRY_MIN_BLOCKS
#define PCR_GEOMETRY_MIN_BLOCKS 1
#endif

constexpr int kThreads = 256;
// Points per lane per chunk, and the resident blocks per SM the geometry
// kernels are compiled for (a register cap).
constexpr int kUnroll = PCR_GEOMETRY_UNROLL;
constexpr int kMinBlocks = PCR_GEOMETRY_MIN_BLOCKS;
// HQ colour pass: above this many runs of equal pixels in a warp row the
// warp adds directly instead of aggregating.
constexpr int kAggregateMaxRuns = 12;

__device__ __forceinline__ unsigned long long make_key(float w, uint32_t idx) {
  return (static_cast<unsigned long long>(__float_as_uint(w)) << 32) | idx;
}

// Walk the point chunks of this warp.  For each chunk, f(r, base, full)
// gets the U records of this lane (slot u holds point base + 32u), and
// `full` as a compile-time flag: true when every slot of the chunk lies
// inside the cloud.  Every lane of the warp calls f the same number of times,
// so f may use warp-collective operations.
template <int U, class F>
__device__ __forceinline__ void for_each_chunk(const uint4* __restrict__ pts, uint32_t n, uint64_t pol, F&& f) {
  const uint64_t warps_per_block = blockDim.x >> 5;
  const uint64_t warp = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  const uint64_t nwarps = gridDim.x * warps_per_block;
  constexpr uint64_t kChunk = 32ull * U;
  const uint64_t nfull = n / kChunk;
  const uint32_t lane = lane_id();
  uint64_t c = warp;
  for (; c < nfull; c += nwarps) {
    const uint32_t base = static_cast<uint32_t>(c * kChunk) + lane;
    uint4 r[U];
#pragma unroll
    for (int u = 0; u < U; ++u) r[u] = load_point_stream(pts + base + 32u * u, pol);
    f(r, base, std::true_type{});
  }
  if (c == nfull && nfull * kChunk < n) {  // the one ragged chunk, if any
    const uint64_t base = c * kChunk + lane;
    uint4 r[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = base + 32ull * u;
      r[u] = (i < n) ? load_point_stream(pts + i, pol) : make_uint4(0u, 0u, 0u, 0u);
    }
    f(r, static_cast<uint32_t>(base), std::false_type{});
  }
}

template <class Full>
__device__ __forceinline__ bool slot_in_range(uint32_t base, int u, uint32_t n, Full) {
  if constexpr (Full::value) {
    return true;
  } else {
    return static_cast<uint64_t>(base) + 32ull * u < n;
  }
}

__device__ __forceinline__ bool project_record(const ViewParams& v, const uint4& r, uint32_t& pix, float& w) {
  return project(v, __uint_as_float(r.x), __uint_as_float(r.y), __uint_as_float(r.z), pix, w);
}

// ---------------------------------------------------------------------------
// Sec. 3.1-3.4: basic key render
// ---------------------------------------------------------------------------

template <int V>
__host__ __device__ constexpr bool reads_early() {
  return V == PCR_VARIANT_EARLYZ || V == PCR_VARIANT_DEDUP_EARLYZ || V == PCR_VARIANT_REDUCE_EARLYZ;
}

// One point slot after projection.  `seen` is this lane's earlier read of
// its pixel (variants with the early test only).
template <int V>
__device__ __forceinline__ void emit_key(unsigned long long* __restrict__ fb, bool vis, uint32_t pix, float w,
                                         uint32_t idx, unsigned long long seen, uint64_t pol) {
  const unsigned long long key = make_key(w, idx);
  if constexpr (V == PCR_VARIANT_ATOMICMIN) {
    // Sec. 3.1: atomicMin(framebuffer[pixelID], point)
    if (vis) red_min_u64(fb + pix, key, pol);
  } else if constexpr (V == PCR_VARIANT_EARLYZ) {
    // Sec. 3.2: only call the atomic when the point is closer than what the
    // buffer (possibly stale, never too small) holds.
    if (vis && key < seen) red_min_u64(fb + pix, key, pol);
  } else if constexpr (V == PCR_VARIANT_DEDUP) {
    // Sec. 3.4: lanes with the same pixel form a group; only the lane with
    // the group's smallest key writes.  Keys reduce on the full 64 bits
    // (depth, then index), so each distinct pixel costs one atomic per warp
    // even when depths tie.  Within a row of the chunk the index grows with
    // the lane, so the smallest index among the smallest depths is the
    // lowest such lane.
    const uint32_t tag = vis ? pix : kNoPixel;
    const uint32_t peers = __match_any_sync(kFullMask, tag);
    const uint32_t hi = vis ? __float_as_uint(w) : 0xFFFFFFFFu;
    const uint32_t hmin = __reduce_min_sync(peers, hi);
    const uint32_t tied = __ballot_sync(kFullMask, hi == hmin) & peers;
    if (vis && lane_id() == static_cast<uint32_t>(__ffs(tied) - 1)) red_min_u64(fb + pix, key, pol);
  } else if constexpr (V == PCR_VARIANT_DEDUP_EARLYZ) {
    // Sec. 3.4 with Sec. 3.2, tests swapped: every visible lane has read its
    // pixel already (cheap, mostly L2 hits); only lanes still closer than the
    // buffer take part in the deduplication, which the whole warp skips when
    // none is left.  A lane dropped by the early test can never hold a
    // pixel's final minimum, so the set of writers still contains it and the
    // buffer is the same.
    const bool want = vis && key < seen;
    const uint32_t active = __ballot_sync(kFullMask, want);
    if (active != 0 && want) {
      const uint32_t peers = __match_any_sync(active, pix);
      const uint32_t hi = __float_as_uint(w);
      const uint32_t hmin = __reduce_min_sync(peers, hi);
      const uint32_t first = __reduce_min_sync(peers, hi == hmin ? lane_id() : 32u);
      if (lane_id() == first) red_min_u64(fb + pix, key, pol);
    }
  } else if constexpr (V == PCR_VARIANT_REDUCE || V == PCR_VARIANT_REDUCE_EARLYZ) {
    // Sec. 3.3: if the whole warp targets one pixel, one lane writes the
    // warp's minimum; otherwise pairs of neighbouring lanes merge when they
    // share a pixel (the smaller key writes).
    const uint32_t tag = vis ? pix : kNoPixel;
    int all_equal = 0;
    __match_all_sync(kFullMask, tag, &all_equal);
    bool write = vis;
    if (all_equal) {
      const uint32_t hi = vis ? __float_as_uint(w) : 0xFFFFFFFFu;
      const uint32_t hmin = __reduce_min_sync(kFullMask, hi);
      const uint32_t tied = __ballot_sync(kFullMask, hi == hmin);
      write = vis && lane_id() == static_cast<uint32_t>(__ffs(tied) - 1);
    } else {
      const uint32_t other_tag = __shfl_xor_sync(kFullMask, tag, 1);
      const unsigned long long other_key = __shfl_xor_sync(kFullMask, key, 1);
      if (other_tag == tag) write = vis && key < other_key;
    }
    if (write && (V == PCR_VARIANT_REDUCE || key < seen)) red_min_u64(fb + pix, key, pol);
  } else {
    // Sec. 5 "just-set": plain store, no depth test; the last writer wins.
    static_assert(V == PCR_VARIANT_JUST_SET, "unknown variant");
    if (vis) {
      asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(fb + pix), "l"(key));
    }
  }
}

// Each chunk runs in three phases so independent memory round trips overlap:
// project all U points, issue all U early reads, then test and write.
template <int V, int U>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_render_basic(const uint4* __restrict__ pts, uint32_t n, ViewParams v,
                                                           unsigned long long* __restrict__ fb) {
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_fb = policy_evict_last();
  for_each_chunk<U>(pts, n, pol_stream, [&](const uint4(&r)[U], uint32_t base, auto full) {
    uint32_t pix[U];
    float w[U];
    bool vis[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      pix[u] = 0;
      w[u] = 0.0f;
      vis[u] = slot_in_range(base, u, n, full) && project_record(v, r[u], pix[u], w[u]);
    }
    unsigned long long seen[U];
#pragma unroll
    for (int u = 0; u < U; ++u) seen[u] = (reads_early<V>() && vis[u]) ? load_relaxed_u64(fb + pix[u]) : 0ull;
#pragma unroll
    for (int u = 0; u < U; ++u) emit_key<V>(fb, vis[u], pix[u], w[u], base + 32u * u, seen[u], pol_fb);
  });
}

// ---------------------------------------------------------------------------
// Sec. 3.5: high-quality passes
// ---------------------------------------------------------------------------

template <int V>
__device__ __forceinline__ void emit_depth(uint32_t* __restrict__ depth, bool vis, uint32_t pix, uint32_t d,
                                           uint32_t seen, uint64_t pol) {
  if constexpr (V == PCR_VARIANT_ATOMICMIN) {
    if (vis) red_min_u32(depth + pix, d, pol);
  } else if constexpr (V == PCR_VARIANT_EARLYZ) {
    if (vis && d < seen) red_min_u32(depth + pix, d, pol);
  } else if constexpr (V == PCR_VARIANT_DEDUP) {
    // The group's minimum can be written by any of its lanes: the lowest.
    const uint32_t tag = vis ? pix : kNoPixel;
    const uint32_t peers = __match_any_sync(kFullMask, tag);
    const uint32_t dmin = __reduce_min_sync(peers, vis ? d : 0xFFFFFFFFu);
    if (vis && lane_id() == static_cast<uint32_t>(__ffs(peers) - 1)) red_min_u32(depth + pix, dmin, pol);
  } else {
    // Early test first, then deduplicate the lanes that are still closer.
    static_assert(V == PCR_VARIANT_DEDUP_EARLYZ, "unknown depth variant");
    const bool want = vis && d < seen;
    const uint32_t active = __ballot_sync(kFullMask, want);
    if (active != 0 && want) {
      const uint32_t peers = __match_any_sync(active, pix);
      const uint32_t dmin = __reduce_min_sync(peers, d);
      if (lane_id() == static_cast<uint32_t>(__ffs(peers) - 1)) red_min_u32(depth + pix, dmin, pol);
    }
  }
}

template <int V, int U>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_hq_depth(const uint4* __restrict__ pts, uint32_t n, ViewParams v,
                                                       uint32_t* __restrict__ depth) {
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_fb = policy_evict_last();
  constexpr bool kEarly = V == PCR_VARIANT_EARLYZ || V == PCR_VARIANT_DEDUP_EARLYZ;
  for_each_chunk<U>(pts, n, pol_stream, [&](const uint4(&r)[U], uint32_t base, auto full) {
    uint32_t pix[U];
    float w[U];
    bool vis[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      pix[u] = 0;
      w[u] = 0.0f;
      vis[u] = slot_in_range(base, u, n, full) && project_record(v, r[u], pix[u], w[u]);
    }
    uint32_t seen[U];
#pragma unroll
    for (int u = 0; u < U; ++u) seen[u] = (kEarly && vis[u]) ? load_relaxed_u32(depth + pix[u]) : 0u;
#pragma unroll
    for (int u = 0; u < U; ++u) emit_depth<V>(depth, vis[u], pix[u], __float_as_uint(w[u]), seen[u], pol_fb);
  });
}

// Colour pass (Listing "hqs_render"): a visible point contributes when
// w <= depth * factor.  With AGG, lanes that contribute to the same pixel
// first sum their colours inside the warp (at most 32 * 255 per channel,
// so r | g << 16 and b | count << 16 cannot carry), then one lane adds.
template <bool AGG>
__device__ __forceinline__ void emit_color(unsigned long long* __restrict__ rg, unsigned long long* __restrict__ ba,
                                           bool contrib, uint32_t pix, uint32_t rgba, uint64_t pol) {
  const uint32_t cr = rgba & 0xFFu;
  const uint32_t cg = (rgba >> 8) & 0xFFu;
  const uint32_t cb = (rgba >> 16) & 0xFFu;
  if constexpr (!AGG) {
    if (contrib) {
      red_add_u64(rg + pix, (static_cast<unsigned long long>(cr) << 32) | cg, pol);
      red_add_u64(ba + pix, (static_cast<unsigned long long>(cb) << 32) | 1ull, pol);
    }
  } else {
    // Aggregate only when the contributing lanes share pixels: count the
    // runs of equal pixels among neighbouring lanes (cheap), and fall back
    // to plain adds when the warp's pixels are mostly distinct (shuffled
    // orders), where matching would cost more than it saves.
    const uint32_t tag = contrib ? pix : kNoPixel;
    const uint32_t active = __ballot_sync(kFullMask, contrib);
    const uint32_t prev = __shfl_up_sync(kFullMask, tag, 1);
    const uint32_t starts = __ballot_sync(kFullMask, contrib && (lane_id() == 0 || prev != tag));
    if (__popc(starts) > kAggregateMaxRuns) {
      if (contrib) {
        red_add_u64(rg + pix, (static_cast<unsigned long long>(cr) << 32) | cg, pol);
        red_add_u64(ba + pix, (static_cast<unsigned long long>(cb) << 32) | 1ull, pol);
      }
    } else if (contrib) {
      const uint32_t peers = __match_any_sync(active, pix);
      const uint32_t s_rg = __reduce_add_sync(peers, cr | (cg << 16));
      const uint32_t s_bc = __reduce_add_sync(peers, cb | (1u << 16));
      if (lane_id() == static_cast<uint32_t>(__ffs(peers) - 1)) {
        red_add_u64(rg + pix, (static_cast<unsigned long long>(s_rg & 0xFFFFu) << 32) | (s_rg >> 16), pol);
        red_add_u64(ba + pix, (static_cast<unsigned long long>(s_bc & 0xFFFFu) << 32) | (s_bc >> 16), pol);
      }
    }
  }
}

template <bool AGG, int U>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_hq_color(const uint4* __restrict__ pts, uint32_t n, ViewParams v,
                                                       float factor, const uint32_t* __restrict__ depth,
                                                       unsigned long long* __restrict__ rg,
                                                       unsigned long long* __restrict__ ba) {
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_fb = policy_evict_last();
  for_each_chunk<U>(pts, n, pol_stream, [&](const uint4(&r)[U], uint32_t base, auto full) {
    uint32_t pix[U];
    float w[U];
    bool vis[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      pix[u] = 0;
      w[u] = 0.0f;
      vis[u] = slot_in_range(base, u, n, full) && project_record(v, r[u], pix[u], w[u]);
    }
    uint32_t d[U];
#pragma unroll
    for (int u = 0; u < U; ++u) d[u] = vis[u] ? __ldg(depth + pix[u]) : 0u;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool contrib = vis[u] && w[u] <= __fmul_rn(__uint_as_float(d[u]), factor);
      emit_color<AGG>(rg, ba, contrib, pix[u], r[u].w, pol_fb);
    }
  });
}

// Sec. 3.5.1, "HQS1R": one 64-bit add per contributing lane, or per group of
// same-pixel lanes with AGG, into the primary word
//   r << 50 | g << 36 | b << 22 | count      (14, 14, 14, 22 bits).
// The paper packs 16-16-16-16 and notes that the pattern must change when
// more than about 65k adds to one pixel can be in flight at once; on a GB300
// that many can (152 SMs x 2048 threads x 4 slots), so the count gets 22
// bits (about 4.2M of margin) and a word holds at most kHq1rLimit = 64
// points, whose channel sums (at most 64 * 255) fit 14 bits.  Group sums stay
// below 32 * 255.  Let c be the count the word held before an add of k
// points.  If c + k > kHq1rLimit the add does not stay in the word: when
// c <= kHq1rLimit this add crossed the limit, so it resets the word and moves
// the c points it held (no field has carried) together with its own k points
// into the 32-bit fallback sums; when c > kHq1rLimit the word is already
// past the limit (its owner is about to reset it, discarding this add's bits)
// and the add goes to the fallback.  Each slot's atomic is issued before any
// slot waits on a returned value.
constexpr uint32_t kHq1rLimit = 64;
constexpr int kHq1rShiftR = 50, kHq1rShiftG = 36, kHq1rShiftB = 22;
constexpr unsigned long long kHq1rChannelMask = 0x3FFFull;
constexpr unsigned long long kHq1rCountMask = 0x3FFFFFull;

template <bool AGG, int U>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    k_hq1r_color(const uint4* __restrict__ pts, uint32_t n, ViewParams v, float factor,
                 const uint32_t* __restrict__ depth, unsigned long long* __restrict__ primary,
                 unsigned long long* __restrict__ rg, unsigned long long* __restrict__ ba) {
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_fb = policy_evict_last();
  for_each_chunk<U>(pts, n, pol_stream, [&](const uint4(&r)[U], uint32_t base, auto full) {
    uint32_t pix[U];
    float w[U];
    bool vis[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      pix[u] = 0;
      w[u] = 0.0f;
      vis[u] = slot_in_range(base, u, n, full) && project_record(v, r[u], pix[u], w[u]);
    }
    uint32_t d[U];
#pragma unroll
    for (int u = 0; u < U; ++u) d[u] = vis[u] ? __ldg(depth + pix[u]) : 0u;
    bool mine[U];
    uint32_t sr[U], sg[U], sb[U], k[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool contrib = vis[u] && w[u] <= __fmul_rn(__uint_as_float(d[u]), factor);
      sr[u] = r[u].w & 0xFFu;
      sg[u] = (r[u].w >> 8) & 0xFFu;
      sb[u] = (r[u].w >> 16) & 0xFFu;
      k[u] = 1;
      mine[u] = contrib;
      if constexpr (AGG) {
        const uint32_t tag = contrib ? pix[u] : kNoPixel;
        const uint32_t active = __ballot_sync(kFullMask, contrib);
        const uint32_t prev = __shfl_up_sync(kFullMask, tag, 1);
        const uint32_t starts = __ballot_sync(kFullMask, contrib && (lane_id() == 0 || prev != tag));
        if (__popc(starts) <= kAggregateMaxRuns && contrib) {
          const uint32_t peers = __match_any_sync(active, pix[u]);
          const uint32_t s_rg = __reduce_add_sync(peers, sr[u] | (sg[u] << 16));
          const uint32_t s_bc = __reduce_add_sync(peers, sb[u] | (1u << 16));
          mine[u] = lane_id() == static_cast<uint32_t>(__ffs(peers) - 1);
          sr[u] = s_rg & 0xFFFFu;
          sg[u] = s_rg >> 16;
          sb[u] = s_bc & 0xFFFFu;
          k[u] = s_bc >> 16;
        }
      }
    }
    unsigned long long old[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      old[u] = 0;
      if (mine[u]) {
        const unsigned long long add = (static_cast<unsigned long long>(sr[u]) << kHq1rShiftR) |
                                       (static_cast<unsigned long long>(sg[u]) << kHq1rShiftG) |
                                       (static_cast<unsigned long long>(sb[u]) << kHq1rShiftB) | k[u];
        old[u] = atom_add_u64(primary + pix[u], add, pol_fb);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!mine[u]) continue;
      const uint32_t c = static_cast<uint32_t>(old[u] & kHq1rCountMask);
      if (c + k[u] <= kHq1rLimit) continue;
      uint32_t fr = sr[u], fg = sg[u], fb = sb[u], fk = k[u];
      if (c <= kHq1rLimit) {
        atom_exch_u64(primary + pix[u], 0ull);
        fr += static_cast<uint32_t>((old[u] >> kHq1rShiftR) & kHq1rChannelMask);
        fg += static_cast<uint32_t>((old[u] >> kHq1rShiftG) & kHq1rChannelMask);
        fb += static_cast<uint32_t>((old[u] >> kHq1rShiftB) & kHq1rChannelMask);
        fk += c;
      }
      red_add_u64(rg + pix[u], (static_cast<unsigned long long>(fr) << 32) | fg, pol_fb);
      red_add_u64(ba + pix[u], (static_cast<unsigned long long>(fb) << 32) | fk, pol_fb);
    }
  });
}

// ---------------------------------------------------------------------------
// Clears and resolves (screen passes)
// ---------------------------------------------------------------------------

__global__ void k_fill_u64(unsigned long long* __restrict__ p, uint64_t count, unsigned long long value) {
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
    p[i] = value;
}

__global__ void k_clear_hq(uint32_t* __restrict__ depth, unsigned long long* __restrict__ rg,
                           unsigned long long* __restrict__ ba, uint64_t npx) {
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < npx;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    depth[i] = kInfBits;
    rg[i] = 0ull;
    ba[i] = 0ull;
  }
}

// Sec. 3.1, Listing "resolve": the winning point's colour, looked up through
// the index payload.
__global__ void k_resolve_basic(const unsigned long long* __restrict__ keys, uint64_t npx,
                                const uint32_t* __restrict__ words, uint32_t n, uint32_t background,
                                uint32_t* __restrict__ out) {
  for (uint64_t p = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; p < npx;
       p += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const unsigned long long k = keys[p];
    const uint32_t idx = static_cast<uint32_t>(k);
    uint32_t c = background;
    if (k != kEmptyKey) {
      if (idx < n)
        c = __ldg(words + 4ull * idx + 3);
      else
        atomicOr(&g_error_word, 1u);
    }
    out[p] = c;
  }
}

// Sec. 3.5, Listing "hqs_resolve": truncating average, alpha 255.
__global__ void k_resolve_hq(const unsigned long long* __restrict__ rg, const unsigned long long* __restrict__ ba,
                             uint64_t npx, uint32_t background, uint32_t* __restrict__ out) {
  for (uint64_t p = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; p < npx;
       p += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const unsigned long long s_rg = rg[p];
    const unsigned long long s_ba = ba[p];
    const uint32_t a = static_cast<uint32_t>(s_ba);
    uint32_t c = background;
    if (a != 0) {
      const uint32_t r = min(static_cast<uint32_t>(s_rg >> 32) / a, 255u);
      const uint32_t g = min(static_cast<uint32_t>(s_rg) / a, 255u);
      const uint32_t b = min(static_cast<uint32_t>(s_ba >> 32) / a, 255u);
      c = r | (g << 8) | (b << 16) | 0xFF000000u;
    }
    out[p] = c;
  }
}

// Sec. 3.5.1: average over the primary word's fields plus the fallback sums.
__global__ void k_resolve_hq1r(const unsigned long long* __restrict__ primary, const unsigned long long* __restrict__ rg,
                               const unsigned long long* __restrict__ ba, uint64_t npx, uint32_t background,
                               uint32_t* __restrict__ out) {
  for (uint64_t p = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; p < npx;
       p += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const unsigned long long w1 = primary[p];
    const unsigned long long s_rg = rg[p];
    const unsigned long long s_ba = ba[p];
    const uint32_t a = static_cast<uint32_t>(s_ba) + static_cast<uint32_t>(w1 & kHq1rCountMask);
    uint32_t c = background;
    if (a != 0) {
      const uint32_t sr = static_cast<uint32_t>(s_rg >> 32) + static_cast<uint32_t>((w1 >> kHq1rShiftR) & kHq1rChannelMask);
      const uint32_t sg = static_cast<uint32_t>(s_rg) + static_cast<uint32_t>((w1 >> kHq1rShiftG) & kHq1rChannelMask);
      const uint32_t sb = static_cast<uint32_t>(s_ba >> 32) + static_cast<uint32_t>((w1 >> kHq1rShiftB) & kHq1rChannelMask);
      c = min(sr / a, 255u) | (min(sg / a, 255u) << 8) | (min(sb / a, 255u) << 16) | 0xFF000000u;
    }
    out[p] = c;
  }
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------

template <class K>
int resident_blocks(K kernel) {
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, kThreads, 0) != cudaSuccess || blocks < 1)
    blocks = 1;
  return blocks;
}

// Persistent geometry grid: enough blocks to fill every SM, never more than
// there are chunks.  The resident-block count is cached per kernel.
template <auto K, int U>
dim3 geometry_grid(uint32_t n, const Device& d) {
  static const int resident = resident_blocks(K);
  const uint64_t points_per_block = (kThreads / 32) * 32ull * U;
  const uint64_t need = (static_cast<uint64_t>(n) + points_per_block - 1) / points_per_block;
  const uint64_t full = static_cast<uint64_t>(d.num_sms) * resident;
  return dim3(static_cast<unsigned>(need < full ? (need > 0 ? need : 1) : full));
}

dim3 screen_grid(uint64_t npx, const Device& d) {
  const uint64_t need = (npx + kThreads - 1) / kThreads;
  const uint64_t cap = static_cast<uint64_t>(d.num_sms) * 8;
  return dim3(static_cast<unsigned>(need < cap ? (need > 0 ? need : 1) : cap));
}

template <int V>
cudaError_t launch_basic_v(const uint4* pts, uint32_t n, const ViewParams& v, unsigned long long* keys, cudaStream_t s,
                           const Device& d) {
  constexpr auto k = k_render_basic<V, kUnroll>;
  k<<<geometry_grid<k, kUnroll>(n, d), kThreads, 0, s>>>(pts, n, v, keys);
  return cudaGetLastError();
}

template <int V>
cudaError_t launch_depth_v(const uint4* pts, uint32_t n, const ViewParams& v, uint32_t* depth, cudaStream_t s,
                           const Device& d) {
  constexpr auto k = k_hq_depth<V, kUnroll>;
  k<<<geometry_grid<k, kUnroll>(n, d), kThreads, 0, s>>>(pts, n, v, depth);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fill_u64(unsigned long long* p, uint64_t count, unsigned long long value, cudaStream_t s,
                            const Device& d) {
  if (count == 0) return cudaSuccess;
  k_fill_u64<<<screen_grid(count, d), kThreads, 0, s>>>(p, count, value);
  return cudaGetLastError();
}

cudaError_t launch_clear_hq(uint32_t* depth, unsigned long long* rg, unsigned long long* ba, uint64_t npx,
                            cudaStream_t s, const Device& d) {
  if (npx == 0) return cudaSuccess;
  k_clear_hq<<<screen_grid(npx, d), kThreads, 0, s>>>(depth, rg, ba, npx);
  return cudaGetLastError();
}

cudaError_t launch_render_basic(int variant, const uint4* pts, uint32_t n, const ViewParams& v,
                                unsigned long long* keys, cudaStream_t s, const Device& d) {
  if (n == 0) return cudaSuccess;
  switch (variant) {
    case PCR_VARIANT_ATOMICMIN: return launch_basic_v<PCR_VARIANT_ATOMICMIN>(pts, n, v, keys, s, d);
    case PCR_VARIANT_EARLYZ: return launch_basic_v<PCR_VARIANT_EARLYZ>(pts, n, v, keys, s, d);
    case PCR_VARIANT_DEDUP: return launch_basic_v<PCR_VARIANT_DEDUP>(pts, n, v, keys, s, d);
    case PCR_VARIANT_DEDUP_EARLYZ: return launch_basic_v<PCR_VARIANT_DEDUP_EARLYZ>(pts, n, v, keys, s, d);
    case PCR_VARIANT_REDUCE: return launch_basic_v<PCR_VARIANT_REDUCE>(pts, n, v, keys, s, d);
    case PCR_VARIANT_REDUCE_EARLYZ: return launch_basic_v<PCR_VARIANT_REDUCE_EARLYZ>(pts, n, v, keys, s, d);
    case PCR_VARIANT_JUST_SET: return launch_basic_v<PCR_VARIANT_JUST_SET>(pts, n, v, keys, s, d);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_hq_depth(int variant, const uint4* pts, uint32_t n, const ViewParams& v, uint32_t* depth,
                            cudaStream_t s, const Device& d) {
  if (n == 0) return cudaSuccess;
  switch (variant) {
    case PCR_VARIANT_ATOMICMIN: return launch_depth_v<PCR_VARIANT_ATOMICMIN>(pts, n, v, depth, s, d);
    case PCR_VARIANT_EARLYZ: return launch_depth_v<PCR_VARIANT_EARLYZ>(pts, n, v, depth, s, d);
    case PCR_VARIANT_DEDUP: return launch_depth_v<PCR_VARIANT_DEDUP>(pts, n, v, depth, s, d);
    case PCR_VARIANT_DEDUP_EARLYZ: return launch_depth_v<PCR_VARIANT_DEDUP_EARLYZ>(pts, n, v, depth, s, d);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_hq_color(int variant, const uint4* pts, uint32_t n, const ViewParams& v, float depth_factor,
                            const uint32_t* depth, unsigned long long* rg, unsigned long long* ba, cudaStream_t s,
                            const Device& d) {
  if (n == 0) return cudaSuccess;
  if (variant == PCR_VARIANT_DEDUP || variant == PCR_VARIANT_DEDUP_EARLYZ) {
    constexpr auto k = k_hq_color<true, kUnroll>;
    k<<<geometry_grid<k, kUnroll>(n, d), kThreads, 0, s>>>(pts, n, v, depth_factor, depth, rg, ba);
  } else {
    constexpr auto k = k_hq_color<false, kUnroll>;
    k<<<geometry_grid<k, kUnroll>(n, d), kThreads, 0, s>>>(pts, n, v, depth_factor, depth, rg, ba);
  }
  return cudaGetLastError();
}

cudaError_t launch_hq1r_color(int variant, const uint4* pts, uint32_t n, const ViewParams& v, float depth_factor,
                              const uint32_t* depth, unsigned long long* primary, unsigned long long* rg,
                              unsigned long long* ba, cudaStream_t s, const Device& d) {
  if (n == 0) return cudaSuccess;
  if (variant == PCR_VARIANT_DEDUP || variant == PCR_VARIANT_DEDUP_EARLYZ) {
    constexpr auto k = k_hq1r_color<true, kUnroll>;
    k<<<geometry_grid<k, kUnroll>(n, d), kThreads, 0, s>>>(pts, n, v, depth_factor, depth, primary, rg, ba);
  } else {
    constexpr auto k = k_hq1r_color<false, kUnroll>;
    k<<<geometry_grid<k, kUnroll>(n, d), kThreads, 0, s>>>(pts, n, v, depth_factor, depth, primary, rg, ba);
  }
  return cudaGetLastError();
}

cudaError_t launch_resolve_hq1r(const unsigned long long* primary, const unsigned long long* rg,
                                const unsigned long long* ba, uint64_t npx, uint32_t background, uint32_t* out,
                                cudaStream_t s, const Device& d) {
  if (npx == 0) return cudaSuccess;
  k_resolve_hq1r<<<screen_grid(npx, d), kThreads, 0, s>>>(primary, rg, ba, npx, background, out);
  return cudaGetLastError();
}

cudaError_t launch_resolve_basic(const unsigned long long* keys, uint64_t npx, const uint4* pts, uint32_t n,
                                 uint32_t background, uint32_t* out, cudaStream_t s, const Device& d) {
  if (npx == 0) return cudaSuccess;
  k_resolve_basic<<<screen_grid(npx, d), kThreads, 0, s>>>(keys, npx, reinterpret_cast<const uint32_t*>(pts), n,
                                                           background, out);
  return cudaGetLastError();
}

cudaError_t launch_resolve_hq(const unsigned long long* rg, const unsigned long long* ba, uint64_t npx,
                              uint32_t background, uint32_t* out, cudaStream_t s, const Device& d) {
  if (npx == 0) return cudaSuccess;
  k_resolve_hq<<<screen_grid(npx, d), kThreads, 0, s>>>(rg, ba, npx, background, out);
  return cudaGetLastError();
}

cudaError_t read_and_clear_error_word(uint32_t* out, cudaStream_t s) {
  uint32_t zero = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_error_word, sizeof(uint32_t), 0, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbolAsync(g_error_word, &zero, sizeof(uint32_t), 0, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

}  // namespace pcr
