// Per-point building blocks shared by the geometry kernels (render.cu) and
// the batched kernels (batch.cu): the chunk walk and the per-variant writes
// of Sec. 3.1-3.5.
#pragma once

#include <cstdint>
#include <type_traits>

#include "../../include/pcr.h"
#include "common.cuh"

namespace pcr {
namespace geom {

// HQ colour pass: above this many runs of equal pixels in a warp row the
// warp adds directly instead of aggregating.
constexpr int kAggregateMaxRuns = 12;

// Key payloads (Sec. 3.1): the point index below the depth bits (the
// colour is looked up in the resolve), or, as Listing "basic" prints it, the
// 24-bit colour below depth bits shifted by 24.
enum Payload { kPayloadIndex = 0, kPayloadRgb = 1 };

__device__ __forceinline__ unsigned long long make_key(float w, uint32_t idx) {
  return (static_cast<unsigned long long>(__float_as_uint(w)) << 32) | idx;
}

template <int P>
__device__ __forceinline__ unsigned long long make_payload_key(float w, uint32_t payload) {
  if constexpr (P == kPayloadRgb) {
    return (static_cast<unsigned long long>(__float_as_uint(w)) << 24) | (payload & 0xFFFFFFu);
  } else {
    return make_key(w, payload);
  }
}

// The lane of `tied` (the lanes of a group whose depth equals the group's
// minimum; `mine` says whether this lane is one of them) that holds the
// group's smallest key.  With the index payload the index grows with the
// lane inside a row of the chunk, so it is the lowest tied lane; with the
// colour payload it is the lowest tied lane with the smallest colour, found
// by the tied lanes alone (others get 32, no lane).
template <int P>
__device__ __forceinline__ uint32_t min_key_lane(uint32_t tied, bool mine, uint32_t payload) {
  if constexpr (P == kPayloadRgb) {
    if (!mine) return 32u;
    const uint32_t c = payload & 0xFFFFFFu;
    const uint32_t cmin = __reduce_min_sync(tied, c);
    return static_cast<uint32_t>(__ffs(__ballot_sync(tied, c == cmin)) - 1);
  } else {
    return static_cast<uint32_t>(__ffs(tied) - 1);
  }
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

// One point slot after projection.  `payload` is the point index or its
// rgba word (P); `seen` is this lane's earlier read of its pixel (variants
// with the early test only).
template <int V, int P = kPayloadIndex>
__device__ __forceinline__ void emit_key(unsigned long long* __restrict__ fb, bool vis, uint32_t pix, float w,
                                         uint32_t payload, unsigned long long seen, uint64_t pol) {
  const unsigned long long key = make_payload_key<P>(w, payload);
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
    // (depth, then payload), so each distinct pixel costs one atomic per
    // warp even when depths tie.
    const uint32_t tag = vis ? pix : kNoPixel;
    const uint32_t peers = __match_any_sync(kFullMask, tag);
    const uint32_t hi = vis ? __float_as_uint(w) : 0xFFFFFFFFu;
    const uint32_t hmin = __reduce_min_sync(peers, hi);
    const uint32_t tied = __ballot_sync(kFullMask, hi == hmin) & peers;
    const uint32_t first = min_key_lane<P>(tied, hi == hmin, payload);
    if (vis && lane_id() == first) red_min_u64(fb + pix, key, pol);
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
      uint32_t first;
      if constexpr (P == kPayloadRgb) {
        const uint32_t tied = __ballot_sync(peers, hi == hmin);
        first = min_key_lane<P>(tied, hi == hmin, payload);
      } else {
        first = __reduce_min_sync(peers, hi == hmin ? lane_id() : 32u);
      }
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
      write = vis && lane_id() == min_key_lane<P>(tied, hi == hmin, payload);
    } else {
      const uint32_t other_tag = __shfl_xor_sync(kFullMask, tag, 1);
      const unsigned long long other_key = __shfl_xor_sync(kFullMask, key, 1);
      if (other_tag == tag) {
        // colour keys of two points can be equal: the even lane keeps it
        write = vis && (key < other_key || (P == kPayloadRgb && key == other_key && (lane_id() & 1u) == 0u));
      }
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

// Colour pass (Listing "hqs_render"): whether the warp sums its colours
// before adding, decided once per chunk from its first row of points: the
// runs of equal pixels among neighbouring contributing lanes.  With at most
// kAggregateMaxRuns runs (coherent orders: neighbours share pixels) the warp
// aggregates; otherwise (shuffled orders) matching would cost more than it
// saves.  The rows of a chunk are 32 points apart in the same order, so the
// first row speaks for the others.  Warp-uniform.
__device__ __forceinline__ bool aggregate_chunk(bool contrib0, uint32_t pix0) {
  const uint32_t tag = contrib0 ? pix0 : kNoPixel;
  const uint32_t prev = __shfl_up_sync(kFullMask, tag, 1);
  const uint32_t starts = __ballot_sync(kFullMask, contrib0 && (lane_id() == 0 || prev != tag));
  return __popc(starts) <= kAggregateMaxRuns;
}

// A visible point contributes when w <= depth * factor, adding (r << 32 | g)
// and (b << 32 | 1).  With `agg` (warp-uniform), lanes that contribute to
// the same pixel first sum their colours inside the warp (at most 32 * 255
// per channel, so r | g << 16 and b | count << 16 cannot carry), then one
// lane adds.
__device__ __forceinline__ void emit_color(unsigned long long* __restrict__ rg, unsigned long long* __restrict__ ba,
                                           bool contrib, uint32_t pix, uint32_t rgba, uint64_t pol, bool agg) {
  // r | g << 16 and b | 1 << 16, each one byte permute of the rgba word
  uint32_t s_rg = __byte_perm(rgba, 0u, 0x4140u);
  uint32_t s_bc = __byte_perm(rgba, 0x100u, 0x4542u);
  bool add = contrib;
  if (agg) {
    const uint32_t active = __ballot_sync(kFullMask, contrib);
    if (contrib) {
      const uint32_t peers = __match_any_sync(active, pix);
      s_rg = __reduce_add_sync(peers, s_rg);
      s_bc = __reduce_add_sync(peers, s_bc);
      add = lane_id() == static_cast<uint32_t>(__ffs(peers) - 1);
    }
  }
  if (add) {
    red_add_u64(rg + pix, (static_cast<unsigned long long>(s_rg & 0xFFFFu) << 32) | (s_rg >> 16), pol);
    red_add_u64(ba + pix, (static_cast<unsigned long long>(s_bc & 0xFFFFu) << 32) | (s_bc >> 16), pol);
  }
}

}  // namespace geom
}  // namespace pcr
