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

#include "../../include/pcr.h"
#include "common.cuh"
#include "launch.h"

namespace pcr {

namespace {

__device__ uint32_t g_error_word;

constexpr int kThreads = 256;
constexpr int kUnroll = 4;

__device__ __forceinline__ unsigned long long make_key(float w, uint32_t idx) {
  return (static_cast<unsigned long long>(__float_as_uint(w)) << 32) | idx;
}

// Walk the point chunks of this warp and call f(record, index, in_range) for
// each slot; every lane of the warp calls f the same number of times, so f
// may use warp-collective operations.
template <int U, class F>
__device__ __forceinline__ void for_each_point(const uint4* __restrict__ pts, uint32_t n, uint64_t pol, F&& f) {
  const uint64_t warps_per_block = blockDim.x >> 5;
  const uint64_t warp = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  const uint64_t nwarps = gridDim.x * warps_per_block;
  const uint64_t chunk = 32ull * U;
  const uint64_t nchunks = (static_cast<uint64_t>(n) + chunk - 1) / chunk;
  const uint32_t lane = lane_id();
  for (uint64_t c = warp; c < nchunks; c += nwarps) {
    const uint64_t base = c * chunk + lane;
    uint4 r[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = base + 32ull * u;
      r[u] = (i < n) ? load_point_stream(pts + i, pol) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = base + 32ull * u;
      f(r[u], static_cast<uint32_t>(i), i < n);
    }
  }
}

__device__ __forceinline__ bool project_record(const ViewParams& v, const uint4& r, bool in_range, uint32_t& pix,
                                               float& w) {
  if (!in_range) return false;
  return project(v, __uint_as_float(r.x), __uint_as_float(r.y), __uint_as_float(r.z), pix, w);
}

// ---------------------------------------------------------------------------
// Sec. 3.1-3.4: basic key render
// ---------------------------------------------------------------------------

template <int V>
__device__ __forceinline__ void emit_key(unsigned long long* __restrict__ fb, bool vis, uint32_t pix, float w,
                                         uint32_t idx, uint64_t pol) {
  const unsigned long long key = make_key(w, idx);
  if constexpr (V == PCR_VARIANT_ATOMICMIN) {
    // Sec. 3.1: atomicMin(framebuffer[pixelID], point)
    if (vis) red_min_u64(fb + pix, key, pol);
  } else if constexpr (V == PCR_VARIANT_EARLYZ) {
    // Sec. 3.2: only call the atomic when the point is closer than what the
    // buffer (possibly stale, never too small) holds.
    if (vis && key < load_relaxed_u64(fb + pix)) red_min_u64(fb + pix, key, pol);
  } else if constexpr (V == PCR_VARIANT_DEDUP || V == PCR_VARIANT_DEDUP_EARLYZ) {
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
    if (vis && lane_id() == static_cast<uint32_t>(__ffs(tied) - 1)) {
      if (V == PCR_VARIANT_DEDUP || key < load_relaxed_u64(fb + pix)) red_min_u64(fb + pix, key, pol);
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
    if (write) {
      if (V == PCR_VARIANT_REDUCE || key < load_relaxed_u64(fb + pix)) red_min_u64(fb + pix, key, pol);
    }
  } else {
    // Sec. 5 "just-set": plain store, no depth test; the last writer wins.
    static_assert(V == PCR_VARIANT_JUST_SET, "unknown variant");
    if (vis) {
      asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(fb + pix), "l"(key));
    }
  }
}

template <int V, int U>
__global__ void __launch_bounds__(kThreads) k_render_basic(const uint4* __restrict__ pts, uint32_t n, ViewParams v,
                                                           unsigned long long* __restrict__ fb) {
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_fb = policy_evict_last();
  for_each_point<U>(pts, n, pol_stream, [&](const uint4& r, uint32_t idx, bool in_range) {
    uint32_t pix = 0;
    float w = 0.0f;
    const bool vis = project_record(v, r, in_range, pix, w);
    emit_key<V>(fb, vis, pix, w, idx, pol_fb);
  });
}

// ---------------------------------------------------------------------------
// Sec. 3.5: high-quality passes
// ---------------------------------------------------------------------------

template <int V>
__device__ __forceinline__ void emit_depth(uint32_t* __restrict__ depth, bool vis, uint32_t pix, uint32_t d,
                                           uint64_t pol) {
  if constexpr (V == PCR_VARIANT_ATOMICMIN) {
    if (vis) red_min_u32(depth + pix, d, pol);
  } else if constexpr (V == PCR_VARIANT_EARLYZ) {
    if (vis && d < load_relaxed_u32(depth + pix)) red_min_u32(depth + pix, d, pol);
  } else {
    // The group's minimum can be written by any of its lanes: the lowest.
    static_assert(V == PCR_VARIANT_DEDUP || V == PCR_VARIANT_DEDUP_EARLYZ, "unknown depth variant");
    const uint32_t tag = vis ? pix : kNoPixel;
    const uint32_t peers = __match_any_sync(kFullMask, tag);
    const uint32_t dmin = __reduce_min_sync(peers, vis ? d : 0xFFFFFFFFu);
    if (vis && lane_id() == static_cast<uint32_t>(__ffs(peers) - 1)) {
      if (V == PCR_VARIANT_DEDUP || dmin < load_relaxed_u32(depth + pix)) red_min_u32(depth + pix, dmin, pol);
    }
  }
}

template <int V, int U>
__global__ void __launch_bounds__(kThreads) k_hq_depth(const uint4* __restrict__ pts, uint32_t n, ViewParams v,
                                                       uint32_t* __restrict__ depth) {
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_fb = policy_evict_last();
  for_each_point<U>(pts, n, pol_stream, [&](const uint4& r, uint32_t, bool in_range) {
    uint32_t pix = 0;
    float w = 0.0f;
    const bool vis = project_record(v, r, in_range, pix, w);
    emit_depth<V>(depth, vis, pix, __float_as_uint(w), pol_fb);
  });
}

// Colour pass (Listing "hqs_render"): a visible point contributes when
// w <= depth * factor.  With AGG, lanes that contribute to the same pixel
// first sum their colours inside the warp (at most 32 * 255 per channel,
// so r | g << 16 and b | count << 16 cannot carry), then one lane adds.
template <bool AGG, int U>
__global__ void __launch_bounds__(kThreads) k_hq_color(const uint4* __restrict__ pts, uint32_t n, ViewParams v,
                                                       float factor, const uint32_t* __restrict__ depth,
                                                       unsigned long long* __restrict__ rg,
                                                       unsigned long long* __restrict__ ba) {
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_fb = policy_evict_last();
  for_each_point<U>(pts, n, pol_stream, [&](const uint4& r, uint32_t, bool in_range) {
    uint32_t pix = 0;
    float w = 0.0f;
    bool contrib = project_record(v, r, in_range, pix, w);
    if (contrib) {
      const float limit = __fmul_rn(__uint_as_float(__ldg(depth + pix)), factor);
      contrib = w <= limit;
    }
    const uint32_t cr = r.w & 0xFFu;
    const uint32_t cg = (r.w >> 8) & 0xFFu;
    const uint32_t cb = (r.w >> 16) & 0xFFu;
    if constexpr (!AGG) {
      if (contrib) {
        red_add_u64(rg + pix, (static_cast<unsigned long long>(cr) << 32) | cg, pol_fb);
        red_add_u64(ba + pix, (static_cast<unsigned long long>(cb) << 32) | 1ull, pol_fb);
      }
    } else {
      const uint32_t tag = contrib ? pix : kNoPixel;
      const uint32_t peers = __match_any_sync(kFullMask, tag);
      const uint32_t s_rg = __reduce_add_sync(peers, contrib ? (cr | (cg << 16)) : 0u);
      const uint32_t s_bc = __reduce_add_sync(peers, contrib ? (cb | (1u << 16)) : 0u);
      if (contrib && lane_id() == static_cast<uint32_t>(__ffs(peers) - 1)) {
        red_add_u64(rg + pix, (static_cast<unsigned long long>(s_rg & 0xFFFFu) << 32) | (s_rg >> 16), pol_fb);
        red_add_u64(ba + pix, (static_cast<unsigned long long>(s_bc & 0xFFFFu) << 32) | (s_bc >> 16), pol_fb);
      }
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
