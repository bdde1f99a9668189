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

// Depth bits and payload of a key.
template <int P>
__device__ __forceinline__ uint32_t key_depth(unsigned long long key) {
  return static_cast<uint32_t>(key >> (P == kPayloadRgb ? 24 : 32));
}
template <int P>
__device__ __forceinline__ uint32_t key_payload(unsigned long long key) {
  return static_cast<uint32_t>(key) & (P == kPayloadRgb ? 0xFFFFFFu : 0xFFFFFFFFu);
}

// The lane of `tied` (the lanes of a group whose depth equals the group's
// minimum; `mine` says whether this lane is one of them) that holds the
// group's smallest key.  With the index payload the indices a row holds grow
// with the lane, so it is the lowest tied lane; with the
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

// Chunks of 32 * U consecutive points, in one of two layouts:
//   kInterleaved: slot u of lane l holds point c * 32U + l + 32u.  Each
//     load instruction covers 512 contiguous bytes, and a row (one slot of
//     every lane) is 32 neighbouring points.  The key and depth passes use
//     it: the early reads of a row then meet few distinct pixels.
//   kConsecutive: slot u of lane l holds point c * 32U + U l + u.  Each lane
//     takes U neighbouring points, so points that share a pixel in a
//     coherent vertex order mostly meet inside one lane, where merging them
//     costs no warp-wide operation.  The grouped colour passes use it.  With V8
//     (the buffer 32-byte aligned, U even) a lane loads its records as U / 2
//     32-byte vectors; a warp's loads together read the chunk's bytes once.
enum Layout { kInterleaved = 0, kConsecutive = 1 };

template <int U, int L>
__device__ __forceinline__ uint32_t slot_index(uint32_t base, int u) {
  return base + static_cast<uint32_t>(L == kConsecutive ? u : 32 * u);
}

// Walk the point chunks of this warp.  For each chunk, f(r, base, full)
// gets the U records of this lane (slot u holds point slot_index(base, u)),
// and `full` as a compile-time flag: true when every slot of the chunk lies
// inside the cloud.  Every lane of the warp calls f the same number of times,
// so f may use warp-collective operations.
template <int U, int L, bool V8, class F>
__device__ __forceinline__ void for_each_chunk(const uint4* __restrict__ pts, uint32_t n, uint64_t pol, F&& f) {
  static_assert(!V8 || (L == kConsecutive && U % 2 == 0), "32-byte loads take a lane's records in pairs");
  const uint64_t warps_per_block = blockDim.x >> 5;
  const uint64_t warp = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  const uint64_t nwarps = gridDim.x * warps_per_block;
  constexpr uint64_t kChunk = 32ull * U;
  constexpr uint32_t kLaneStep = L == kConsecutive ? U : 1;
  const uint64_t nfull = n / kChunk;
  const uint32_t lane = lane_id();
  uint64_t c = warp;
  for (; c < nfull; c += nwarps) {
    const uint32_t base = static_cast<uint32_t>(c * kChunk) + kLaneStep * lane;
    uint4 r[U];
    if constexpr (V8) {
#pragma unroll
      for (int u = 0; u < U; u += 2) load_pair_stream(pts + base + u, pol, r[u], r[u + 1]);
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) r[u] = load_point_stream(pts + slot_index<U, L>(base, u), pol);
    }
    f(r, base, std::true_type{});
  }
  if (c == nfull && nfull * kChunk < n) {  // the one ragged chunk, if any
    const uint32_t base = static_cast<uint32_t>(c * kChunk) + kLaneStep * lane;
    uint4 r[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = static_cast<uint64_t>(base) + (L == kConsecutive ? u : 32ull * u);
      r[u] = (i < n) ? load_point_stream(pts + i, pol) : make_uint4(0u, 0u, 0u, 0u);
    }
    f(r, base, std::false_type{});
  }
}

template <int U, int L, class Full>
__device__ __forceinline__ bool slot_in_range(uint32_t base, int u, uint32_t n, Full) {
  if constexpr (Full::value) {
    return true;
  } else {
    return static_cast<uint64_t>(base) + (L == kConsecutive ? u : 32ull * u) < n;
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

// One point slot after projection: its key (payload P), and `seen`, this
// lane's earlier read of its pixel (variants with the early test only).
template <int V, int P = kPayloadIndex>
__device__ __forceinline__ bool emit_key(unsigned long long* __restrict__ fb, bool vis, uint32_t pix,
                                         unsigned long long key, unsigned long long seen, uint64_t pol,
                                         bool group = true) {
  if constexpr (V == PCR_VARIANT_ATOMICMIN) {
    // Sec. 3.1: a 64-bit minimum of the key into its pixel's word
    if (vis) red_min_u64(fb + pix, key, pol);
    return vis;
  } else if constexpr (V == PCR_VARIANT_EARLYZ) {
    // Sec. 3.2: only call the atomic when the point is closer than what the
    // buffer (possibly stale, never too small) holds.
    const bool write = vis && key < seen;
    if (write) red_min_u64(fb + pix, key, pol);
    return write;
  } else if constexpr (V == PCR_VARIANT_DEDUP) {
    // Sec. 3.4: lanes with the same pixel form a group; only the lane with
    // the group's smallest key writes.  Keys reduce on the full 64 bits
    // (depth, then payload), so each distinct pixel costs one atomic per
    // warp even when depths tie.  `group` (warp-uniform, see dedup_pays)
    // false: the row's pixels are nearly all distinct, so every visible lane
    // writes without the match, which would find groups of one.
    bool write = vis;
    if (group) {
      const uint32_t tag = vis ? pix : kNoPixel;
      const uint32_t peers = __match_any_sync(kFullMask, tag);
      const uint32_t hi = vis ? key_depth<P>(key) : 0xFFFFFFFFu;
      const uint32_t hmin = __reduce_min_sync(peers, hi);
      const uint32_t tied = __ballot_sync(kFullMask, hi == hmin) & peers;
      const uint32_t first = min_key_lane<P>(tied, hi == hmin, key_payload<P>(key));
      write = vis && lane_id() == first;
    }
    if (write) red_min_u64(fb + pix, key, pol);
    return write;
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
      const uint32_t hi = key_depth<P>(key);
      const uint32_t hmin = __reduce_min_sync(peers, hi);
      uint32_t first;
      if constexpr (P == kPayloadRgb) {
        const uint32_t tied = __ballot_sync(peers, hi == hmin);
        first = min_key_lane<P>(tied, hi == hmin, key_payload<P>(key));
      } else {
        first = __reduce_min_sync(peers, hi == hmin ? lane_id() : 32u);
      }
      if (lane_id() == first) {
        red_min_u64(fb + pix, key, pol);
        return true;
      }
    }
    return false;
  } else if constexpr (V == PCR_VARIANT_REDUCE || V == PCR_VARIANT_REDUCE_EARLYZ) {
    // Sec. 3.3: if the whole warp targets one pixel, one lane writes the
    // warp's minimum; otherwise pairs of neighbouring lanes merge when they
    // share a pixel (the smaller key writes).
    const uint32_t tag = vis ? pix : kNoPixel;
    int all_equal = 0;
    __match_all_sync(kFullMask, tag, &all_equal);
    bool write = vis;
    if (all_equal) {
      const uint32_t hi = vis ? key_depth<P>(key) : 0xFFFFFFFFu;
      const uint32_t hmin = __reduce_min_sync(kFullMask, hi);
      const uint32_t tied = __ballot_sync(kFullMask, hi == hmin);
      write = vis && lane_id() == min_key_lane<P>(tied, hi == hmin, key_payload<P>(key));
    } else {
      const uint32_t other_tag = __shfl_xor_sync(kFullMask, tag, 1);
      const unsigned long long other_key = __shfl_xor_sync(kFullMask, key, 1);
      if (other_tag == tag) {
        // colour keys of two points can be equal: the even lane keeps it
        write = vis && (key < other_key || (P == kPayloadRgb && key == other_key && (lane_id() & 1u) == 0u));
      }
    }
    write = write && (V == PCR_VARIANT_REDUCE || key < seen);
    if (write) red_min_u64(fb + pix, key, pol);
    return write;
  } else {
    // Sec. 5 "just-set": plain store, no depth test; the last writer wins.
    static_assert(V == PCR_VARIANT_JUST_SET, "unknown variant");
    if (vis) {
      asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(fb + pix), "l"(key));
    }
    return vis;
  }
}

// Whether warp deduplication (Sec. 3.4, without the early test) pays in this
// chunk, judged from its first row: the runs of equal pixels among
// neighbouring visible lanes.  With more than kDedupMaxRuns the pixels are
// nearly all distinct (shuffled orders) and the match would find groups of
// one.  Warp-uniform.
constexpr int kDedupMaxRuns = 16;
__device__ __forceinline__ bool dedup_pays(bool vis0, uint32_t pix0) {
  const uint32_t tag = vis0 ? pix0 : kNoPixel;
  const uint32_t prev = __shfl_up_sync(kFullMask, tag, 1);
  const uint32_t starts = __ballot_sync(kFullMask, vis0 && (lane_id() == 0 || prev != tag));
  return __popc(starts) <= kDedupMaxRuns;
}

template <int V>
__device__ __forceinline__ bool emit_depth(uint32_t* __restrict__ depth, bool vis, uint32_t pix, uint32_t d,
                                           uint32_t seen, uint64_t pol) {
  if constexpr (V == PCR_VARIANT_ATOMICMIN) {
    if (vis) red_min_u32(depth + pix, d, pol);
    return vis;
  } else if constexpr (V == PCR_VARIANT_EARLYZ) {
    const bool write = vis && d < seen;
    if (write) red_min_u32(depth + pix, d, pol);
    return write;
  } else if constexpr (V == PCR_VARIANT_DEDUP) {
    // The group's minimum can be written by any of its lanes: the lowest.
    const uint32_t tag = vis ? pix : kNoPixel;
    const uint32_t peers = __match_any_sync(kFullMask, tag);
    const uint32_t dmin = __reduce_min_sync(peers, vis ? d : 0xFFFFFFFFu);
    const bool write = vis && lane_id() == static_cast<uint32_t>(__ffs(peers) - 1);
    if (write) red_min_u32(depth + pix, dmin, pol);
    return write;
  } else {
    // Early test first, then deduplicate the lanes that are still closer.
    static_assert(V == PCR_VARIANT_DEDUP_EARLYZ, "unknown depth variant");
    const bool want = vis && d < seen;
    const uint32_t active = __ballot_sync(kFullMask, want);
    if (active != 0 && want) {
      const uint32_t peers = __match_any_sync(active, pix);
      const uint32_t dmin = __reduce_min_sync(peers, d);
      if (lane_id() == static_cast<uint32_t>(__ffs(peers) - 1)) {
        red_min_u32(depth + pix, dmin, pol);
        return true;
      }
    }
    return false;
  }
}

// Sec. 3.5 colour-pass test: a visible point contributes when
// w <= fl(depth * factor), with the depth its pixel holds after the depth
// pass.  The products of two slots form one paired instruction (each half
// rounded as the scalar product).
template <int U>
__device__ __forceinline__ void contributes(const uint32_t* __restrict__ depth, float factor, const uint32_t (&pix)[U],
                                            const float (&w)[U], const bool (&vis)[U], bool (&contrib)[U]) {
  float d[U], thr[U];
#pragma unroll
  for (int u = 0; u < U; ++u) d[u] = vis[u] ? __uint_as_float(__ldg(depth + pix[u])) : 0.0f;
#pragma unroll
  for (int u = 0; u + 1 < U; u += 2) f2_unpack(f2_mul(f2_pack(d[u], d[u + 1]), f2_bcast(factor)), thr[u], thr[u + 1]);
  if constexpr (U % 2 == 1) thr[U - 1] = __fmul_rn(d[U - 1], factor);
#pragma unroll
  for (int u = 0; u < U; ++u) contrib[u] = vis[u] && w[u] <= thr[u];
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Colour pass grouping (Listing "hqs_render" adds (r << 32 | g) and
// (b << 32 | 1) per contributing point; sums do not depend on grouping).
// With AGG:
//   - a slot whose pixel equals the previous slot's, both contributing,
//     joins that slot's run: the lane sums each run of its U neighbouring
//     points (ALU only);
//   - the run from the lane's slot 0 (when it contributes) is summed over
//     the lanes of the warp whose slot-0 run has the same pixel (one match
//     and two reductions per chunk), and the group's lowest lane adds it;
//   - the lane's other runs add directly.
// Without AGG every contributing point adds on its own.  A group holds at
// most 32 U points: for U <= 8, r | g << 16 and b | count << 16 cannot carry.
// On return, add[u] marks the slots that add s_rg[u] (r | g << 16) and
// s_bc[u] (b | count << 16) at pix[u].
template <int U, bool AGG>
__device__ __forceinline__ void group_colors(const bool (&contrib)[U], const uint32_t (&pix)[U], const uint4 (&r)[U],
                                             uint32_t (&s_rg)[U], uint32_t (&s_bc)[U], bool (&add)[U]) {
  static_assert(U <= 8, "group sums would carry");
#pragma unroll
  for (int u = 0; u < U; ++u) {
    // r | g << 16 and b | 1 << 16, each one byte permute of the rgba word
    s_rg[u] = __byte_perm(r[u].w, 0u, 0x4140u);
    s_bc[u] = __byte_perm(r[u].w, 0x100u, 0x4542u);
    add[u] = contrib[u];
  }
  if constexpr (AGG) {
    bool join[U];
    join[0] = false;
#pragma unroll
    for (int u = 1; u < U; ++u) join[u] = contrib[u] && contrib[u - 1] && pix[u] == pix[u - 1];
#pragma unroll
    for (int u = U - 1; u > 0; --u) {
      if (join[u]) {
        s_rg[u - 1] += s_rg[u];
        s_bc[u - 1] += s_bc[u];
      }
    }
#pragma unroll
    for (int u = 1; u < U; ++u) add[u] = contrib[u] && !join[u];
    // the run from slot 0, over the warp: lanes whose slot 0 does not
    // contribute meet under kNoPixel (never a pixel) and add nothing there
    const uint32_t peers = __match_any_sync(kFullMask, contrib[0] ? pix[0] : kNoPixel);
    s_rg[0] = __reduce_add_sync(peers, s_rg[0]);
    s_bc[0] = __reduce_add_sync(peers, s_bc[0]);
    add[0] = contrib[0] && (peers & lanemask_lt()) == 0u;
  }
}

// Returns how many pairs of adds this lane issued.
template <int U, bool AGG>
__device__ __forceinline__ int emit_colors(unsigned long long* __restrict__ rg, unsigned long long* __restrict__ ba,
                                           const bool (&contrib)[U], const uint32_t (&pix)[U], const uint4 (&r)[U],
                                           uint64_t pol) {
  uint32_t s_rg[U], s_bc[U];
  bool add[U];
  group_colors<U, AGG>(contrib, pix, r, s_rg, s_bc, add);
  int adds = 0;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (add[u]) {
      red_add_u64(rg + pix[u], (static_cast<unsigned long long>(s_rg[u] & 0xFFFFu) << 32) | (s_rg[u] >> 16), pol);
      red_add_u64(ba + pix[u], (static_cast<unsigned long long>(s_bc[u] & 0xFFFFu) << 32) | (s_bc[u] >> 16), pol);
      ++adds;
    }
  }
  return adds;
}

}  // namespace geom
}  // namespace pcr
