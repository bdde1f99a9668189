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
#include "geometry.cuh"
#include "launch.h"

namespace pcr {

namespace {

using namespace geom;

// Device-side error word (PCR_DEVICE_ERROR_* bits), read and cleared by
// pcr_last_device_error.
__device__ uint32_t g_error_word;
constexpr uint32_t kErrorKeyRange = PCR_DEVICE_ERROR_KEY_RANGE;
constexpr uint32_t kErrorWaitTimeout = PCR_DEVICE_ERROR_WAIT_TIMEOUT;

// Debug builds (PCR_DEBUG) count what the single-view geometry kernels send
// to the framebuffers: key writes, depth writes, colour add pairs, and the
// early reads; pcr_debug_counters reads and clears them.  They also check
// every visible slot's pixel against the viewport before any access (a
// failure sets kErrorBounds and drops the slot).  Release builds have
// neither.
#ifdef PCR_DEBUG
constexpr uint32_t kErrorBounds = PCR_DEVICE_ERROR_BOUNDS;
__device__ unsigned long long g_debug_counts[4];
#define PCR_DEBUG_COUNT(k, x)                                                     \
  do {                                                                            \
    if (x) atomicAdd(&g_debug_counts[k], static_cast<unsigned long long>(x));     \
  } while (0)
#else
#define PCR_DEBUG_COUNT(k, x) \
  do {                        \
  } while (0)
#endif

template <int U>
__device__ __forceinline__ void debug_check_pixels(const ViewParams& v, const uint32_t (&pix)[U], bool (&vis)[U]) {
#ifdef PCR_DEBUG
  const uint64_t npx = static_cast<uint64_t>(v.width) * v.height;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (vis[u] && pix[u] >= npx) {
      atomicOr(&g_error_word, kErrorBounds);
      vis[u] = false;
    }
  }
#endif
}

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
// Each chunk runs in three phases so independent memory round trips overlap:
// project all U points, issue all U early reads, then test and write.
// P selects the key payload: the point index, or the 24-bit colour.  The
// kernels are held to 40 registers (6 resident blocks of 256 threads per SM):
// the frame is latency-bound, and one resident block fewer costs more than
// the few instructions the register cap adds.
constexpr int kRenderMinBlocks = kMinBlocks < 6 ? 6 : kMinBlocks;
// The HQ depth and colour passes, HQS1R's included, take the same cap (40
// registers each).
constexpr int kHqMinBlocks = kMinBlocks < 6 ? 6 : kMinBlocks;

template <int V, int U, int P>
__global__ void __launch_bounds__(kThreads, kRenderMinBlocks) k_render_basic(const uint4* __restrict__ pts, uint32_t n, ViewParams v,
                                                           unsigned long long* __restrict__ fb) {
  constexpr int L = kInterleaved;
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_fb = policy_evict_last();
  for_each_chunk<U, L, false>(pts, n, pol_stream, [&](const uint4(&r)[U], uint32_t base, auto full) {
    uint32_t pix[U];
    float w[U];
    bool vis[U];
    project_slots<U>(v, r, pix, w, vis);
#pragma unroll
    for (int u = 0; u < U; ++u) vis[u] = vis[u] && slot_in_range<U, L>(base, u, n, full);
    debug_check_pixels<U>(v, pix, vis);
    unsigned long long seen[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      seen[u] = (reads_early<V>() && vis[u]) ? load_relaxed_u64(fb + pix[u]) : 0ull;
      PCR_DEBUG_COUNT(3, reads_early<V>() && vis[u]);
    }
    const bool group = V != PCR_VARIANT_DEDUP || dedup_pays(vis[0], pix[0]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool wrote = emit_key<V, P>(
          fb, vis[u], pix[u], make_payload_key<P>(w[u], P == kPayloadRgb ? r[u].w : slot_index<U, L>(base, u)),
          seen[u], pol_fb, group);
      PCR_DEBUG_COUNT(0, wrote);
    }
  });
}

// ---------------------------------------------------------------------------
// Sec. 2 and Sec. 5 "busy-loop" (Guenther et al.): lock the pixel with a
// compare-and-swap, update it, unlock; with their early depth test.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t cas_acquire_u32(uint32_t* p, uint32_t expect, uint32_t value) {
  uint32_t old;
  asm volatile("atom.acquire.gpu.global.cas.b32 %0, [%1], %2, %3;" : "=r"(old) : "l"(p), "r"(expect), "r"(value)
               : "memory");
  return old;
}

__device__ __forceinline__ void store_release_u32(uint32_t* p, uint32_t value) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(value) : "memory");
}

__device__ __forceinline__ void store_relaxed_u64(unsigned long long* p, unsigned long long value) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(value) : "memory");
}

// Take the pixel's lock, keep the smaller of the stored and the new key,
// release.  Between attempts the early test is repeated: once the pixel holds
// a key at least as small, this point has nothing left to do.  The spin is
// bounded: it gives up when it has waited longer than limit_ns (by the global
// nanosecond timer), after kBusyMaxAttempts attempts (at least half a second
// of backoff), or when another thread has already given up; it then sets
// kErrorWaitTimeout in the error word and drops this point.  Backoff doubles
// from 32 to 1024 ns between attempts.
constexpr uint32_t kBusyMaxAttempts = 1u << 20;
__device__ __forceinline__ void busy_update(unsigned long long* __restrict__ fb, uint32_t* __restrict__ locks,
                                            uint32_t pix, unsigned long long key, uint64_t limit_ns) {
  uint32_t* lock = locks + pix;
  uint64_t t0 = 0;
  uint32_t backoff = 32;
  for (uint32_t attempt = 0;; ++attempt) {
    if (attempt > 0 && load_relaxed_u64(fb + pix) <= key) return;
    if (cas_acquire_u32(lock, 0u, 1u) == 0u) {
      const unsigned long long cur = load_relaxed_u64(fb + pix);
      if (key < cur) store_relaxed_u64(fb + pix, key);
      store_release_u32(lock, 0u);
      return;
    }
    if (attempt == 0) t0 = global_ns();
    if ((attempt & 7u) == 7u && (attempt >= kBusyMaxAttempts || global_ns() - t0 > limit_ns ||
                                 (load_relaxed_u32(&g_error_word) & kErrorWaitTimeout) != 0u)) {
      atomicOr(&g_error_word, kErrorWaitTimeout);
      return;
    }
    __nanosleep(backoff);
    backoff = backoff < 1024u ? backoff * 2u : 1024u;
  }
}

template <int U>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_render_busy(const uint4* __restrict__ pts, uint32_t n, ViewParams v,
                                                          unsigned long long* __restrict__ fb,
                                                          uint32_t* __restrict__ locks, uint64_t limit_ns) {
  const uint64_t pol_stream = policy_evict_first();
  for_each_chunk<U, kInterleaved, false>(pts, n, pol_stream, [&](const uint4(&r)[U], uint32_t base, auto full) {
    uint32_t pix[U];
    float w[U];
    bool vis[U];
    project_slots<U>(v, r, pix, w, vis);
#pragma unroll
    for (int u = 0; u < U; ++u) vis[u] = vis[u] && slot_in_range<U, kInterleaved>(base, u, n, full);
    debug_check_pixels<U>(v, pix, vis);
    unsigned long long seen[U];
#pragma unroll
    for (int u = 0; u < U; ++u) seen[u] = vis[u] ? load_relaxed_u64(fb + pix[u]) : 0ull;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const unsigned long long key = make_key(w[u], slot_index<U, kInterleaved>(base, u));
      if (vis[u] && key < seen[u]) busy_update(fb, locks, pix[u], key, limit_ns);
    }
  });
}

// ---------------------------------------------------------------------------
// Sec. 3.5: high-quality passes
// ---------------------------------------------------------------------------

template <int V, int U>
__global__ void __launch_bounds__(kThreads, kHqMinBlocks) k_hq_depth(const uint4* __restrict__ pts, uint32_t n, ViewParams v,
                                                       uint32_t* __restrict__ depth) {
  constexpr int L = kInterleaved;
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_fb = policy_evict_last();
  constexpr bool kEarly = V == PCR_VARIANT_EARLYZ || V == PCR_VARIANT_DEDUP_EARLYZ;
  for_each_chunk<U, L, false>(pts, n, pol_stream, [&](const uint4(&r)[U], uint32_t base, auto full) {
    uint32_t pix[U];
    float w[U];
    bool vis[U];
    project_slots<U>(v, r, pix, w, vis);
    uint32_t d[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      vis[u] = vis[u] && slot_in_range<U, L>(base, u, n, full);
      d[u] = __float_as_uint(w[u]);
    }
    debug_check_pixels<U>(v, pix, vis);
    uint32_t seen[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      seen[u] = (kEarly && vis[u]) ? load_relaxed_u32(depth + pix[u]) : 0u;
      PCR_DEBUG_COUNT(3, kEarly && vis[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool wrote = emit_depth<V>(depth, vis[u], pix[u], d[u], seen[u], pol_fb);
      PCR_DEBUG_COUNT(1, wrote);
    }
  });
}

// Colour pass (Listing "hqs_render"): see group_colors.
template <bool AGG, int U, bool V8>
__global__ void __launch_bounds__(kThreads, kHqMinBlocks) k_hq_color(const uint4* __restrict__ pts, uint32_t n, ViewParams v,
                                                       float factor, const uint32_t* __restrict__ depth,
                                                       unsigned long long* __restrict__ rg,
                                                       unsigned long long* __restrict__ ba) {
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_fb = policy_evict_last();
  constexpr int L = AGG ? kConsecutive : kInterleaved;
  for_each_chunk<U, L, V8>(pts, n, pol_stream, [&](const uint4(&r)[U], uint32_t base, auto full) {
    uint32_t pix[U];
    float w[U];
    bool vis[U];
    project_slots<U>(v, r, pix, w, vis);
#pragma unroll
    for (int u = 0; u < U; ++u) vis[u] = vis[u] && slot_in_range<U, L>(base, u, n, full);
    debug_check_pixels<U>(v, pix, vis);
    bool contrib[U];
    contributes<U>(depth, factor, pix, w, vis, contrib);
    const int adds = emit_colors<U, AGG>(rg, ba, contrib, pix, r, pol_fb);
    PCR_DEBUG_COUNT(2, adds);
  });
}

// Sec. 3.5.1, "HQS1R": one 64-bit add per contributing point, or per group
// of same-pixel points with AGG (see group_colors), into the primary word
//   r << 50 | g << 36 | b << 22 | count      (14, 14, 14, 22 bits).
// The paper packs 16-16-16-16 and notes that the pattern must change when
// more than about 65k adds to one pixel can be in flight at once; on a GB300
// that many can (152 SMs x 2048 threads x 4 slots), so the count gets 22
// bits (about 4.2M of margin) and a word holds at most kHq1rLimit = 64
// points, whose channel sums (at most 64 * 255) fit 14 bits.  A group of
// more than kHq1rLimit points (up to 128 with AGG) never touches the word: it
// adds its 32-bit sums to the fallback directly.  Let c be the count the
// word held before an add of k <= kHq1rLimit points: see hq1r_settle.
// Without AGG every contributing point adds to the word.  With AGG only the
// warp group of a lane's slot 0 does (one add in flight per lane), and its
// returned value is settled one chunk later, so the wait overlaps the next
// chunk's loads and projection; the lane's other runs add to the fallback.
constexpr uint32_t kHq1rLimit = 64;
constexpr int kHq1rShiftR = 50, kHq1rShiftG = 36, kHq1rShiftB = 22;
constexpr unsigned long long kHq1rChannelMask = 0x3FFFull;
constexpr unsigned long long kHq1rCountMask = 0x3FFFFFull;

// r << 50 | g << 36 | b << 22 | k, built from 32-bit halves (r, g, b below
// 2^14, k below 2^22).
__device__ __forceinline__ unsigned long long hq1r_word(uint32_t r, uint32_t g, uint32_t b, uint32_t k) {
  const uint32_t hi = (r << (kHq1rShiftR - 32)) | (g << (kHq1rShiftG - 32)) | (b >> (32 - kHq1rShiftB));
  const uint32_t lo = (b << kHq1rShiftB) | k;
  return (static_cast<unsigned long long>(hi) << 32) | lo;
}

__device__ __forceinline__ uint32_t hq1r_field(unsigned long long word, int shift) {
  return static_cast<uint32_t>((word >> shift) & kHq1rChannelMask);
}

// The word of a group from its sums s_rg = r | g << 16, s_bc = b | k << 16
// (k <= kHq1rLimit, so each channel fits its field).
__device__ __forceinline__ unsigned long long hq1r_word(uint32_t s_rg, uint32_t s_bc) {
  return hq1r_word(s_rg & 0xFFFFu, s_rg >> 16, s_bc & 0xFFFFu, s_bc >> 16);
}

// A group's sums straight into the 32-bit fallback sums.
__device__ __forceinline__ void hq1r_fallback(unsigned long long* __restrict__ rg, unsigned long long* __restrict__ ba,
                                              uint32_t pix, uint32_t s_rg, uint32_t s_bc, uint64_t pol) {
  red_add_u64(rg + pix, (static_cast<unsigned long long>(s_rg & 0xFFFFu) << 32) | (s_rg >> 16), pol);
  red_add_u64(ba + pix, (static_cast<unsigned long long>(s_bc & 0xFFFFu) << 32) | (s_bc >> 16), pol);
}

// After an add of a group (sums s_rg, s_bc; k <= kHq1rLimit points) to the
// word at pix returned the word's previous value `old`, holding c points:
// c + k <= kHq1rLimit, the add stays; c <= kHq1rLimit < c + k, this add
// crossed the limit: reset the word and move its c points with this add's k
// to the fallback (no field has carried); c > kHq1rLimit, the word's owner is
// about to reset it, discarding this add's bits: this add to the fallback.
__device__ __forceinline__ void hq1r_settle(unsigned long long* __restrict__ primary,
                                            unsigned long long* __restrict__ rg, unsigned long long* __restrict__ ba,
                                            uint32_t pix, uint32_t s_rg, uint32_t s_bc, unsigned long long old,
                                            uint64_t pol) {
  const uint32_t c = static_cast<uint32_t>(old & kHq1rCountMask);
  uint32_t fr = s_rg & 0xFFFFu, fg = s_rg >> 16, fb = s_bc & 0xFFFFu, fk = s_bc >> 16;
  if (c + fk <= kHq1rLimit) return;
  if (c <= kHq1rLimit) {
    atom_exch_u64(primary + pix, 0ull);
    fr += hq1r_field(old, kHq1rShiftR);
    fg += hq1r_field(old, kHq1rShiftG);
    fb += hq1r_field(old, kHq1rShiftB);
    fk += c;
  }
  red_add_u64(rg + pix, (static_cast<unsigned long long>(fr) << 32) | fg, pol);
  red_add_u64(ba + pix, (static_cast<unsigned long long>(fb) << 32) | fk, pol);
}

// HQS1R's colour pass carries one add per lane into the next chunk; it runs
// at 5 resident blocks (48 registers): at 6 it spills, and it was 2% slower.
#ifndef PCR_HQ1R_MIN_BLOCKS
#define PCR_HQ1R_MIN_BLOCKS 5
#endif
template <bool AGG, int U, bool V8>
__global__ void __launch_bounds__(kThreads, PCR_HQ1R_MIN_BLOCKS)
    k_hq1r_color(const uint4* __restrict__ pts, uint32_t n, ViewParams v, float factor,
                 const uint32_t* __restrict__ depth, unsigned long long* __restrict__ primary,
                 unsigned long long* __restrict__ rg, unsigned long long* __restrict__ ba) {
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_fb = policy_evict_last();
  constexpr int L = AGG ? kConsecutive : kInterleaved;
  // with AGG: the one add to a word a lane has in flight, settled in the
  // next chunk (or after the last)
  bool live = false;
  unsigned long long p_old = 0;
  uint32_t p_pix = 0, p_rg = 0, p_bc = 0;
  for_each_chunk<U, L, V8>(pts, n, pol_stream, [&](const uint4(&r)[U], uint32_t base, auto full) {
    uint32_t pix[U];
    float w[U];
    bool vis[U];
    project_slots<U>(v, r, pix, w, vis);
#pragma unroll
    for (int u = 0; u < U; ++u) vis[u] = vis[u] && slot_in_range<U, L>(base, u, n, full);
    debug_check_pixels<U>(v, pix, vis);
    bool contrib[U];
    contributes<U>(depth, factor, pix, w, vis, contrib);
    bool mine[U];
    uint32_t s_rg[U], s_bc[U];
    group_colors<U, AGG>(contrib, pix, r, s_rg, s_bc, mine);
    if constexpr (AGG) {
      // the previous chunk's add to a word: its previous value has arrived
      // while this chunk loaded and projected
      if (live) hq1r_settle(primary, rg, ba, p_pix, p_rg, p_bc, p_old, pol_fb);
      // the warp group of slot 0 adds to the word when it fits one
      live = mine[0] && (s_bc[0] >> 16) <= kHq1rLimit;
      if (live) {
        p_old = atom_add_u64(primary + pix[0], hq1r_word(s_rg[0], s_bc[0]), pol_fb);
        p_pix = pix[0];
        p_rg = s_rg[0];
        p_bc = s_bc[0];
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (mine[u] && !(u == 0 && live)) hq1r_fallback(rg, ba, pix[u], s_rg[u], s_bc[u], pol_fb);
    } else {
      // one point per add: every add to the word, each settled as soon as
      // all U have been issued
      unsigned long long old[U];
#pragma unroll
      for (int u = 0; u < U; ++u) old[u] = mine[u] ? atom_add_u64(primary + pix[u], hq1r_word(s_rg[u], s_bc[u]), pol_fb) : 0ull;
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (mine[u]) hq1r_settle(primary, rg, ba, pix[u], s_rg[u], s_bc[u], old[u], pol_fb);
    }
  });
  if constexpr (AGG) {
    if (live) hq1r_settle(primary, rg, ba, p_pix, p_rg, p_bc, p_old, pol_fb);
  }
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
        atomicOr(&g_error_word, kErrorKeyRange);
    }
    out[p] = c;
  }
}

// Sec. 3.1, Listing "resolve" for colour-payload keys: the colour is in the
// key's low 24 bits; alpha 255.
__global__ void k_resolve_rgb(const unsigned long long* __restrict__ keys, uint64_t npx, uint32_t background,
                              uint32_t* __restrict__ out) {
  for (uint64_t p = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; p < npx;
       p += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const unsigned long long k = keys[p];
    out[p] = k == kEmptyKey ? background : (static_cast<uint32_t>(k) & 0xFFFFFFu) | 0xFF000000u;
  }
}

__global__ void k_fill_u32(uint32_t* __restrict__ p, uint64_t count, uint32_t value) {
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
    p[i] = value;
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

// 32-byte record-pair loads need an even number of points per lane and a
// 32-byte aligned buffer (the interface promises 16 bytes).
constexpr bool kCanPairLoad = kUnroll % 2 == 0;
bool pairs_aligned(const uint4* pts) { return kCanPairLoad && (reinterpret_cast<uintptr_t>(pts) & 31u) == 0; }

template <int V, int P>
cudaError_t launch_basic_v(const uint4* pts, uint32_t n, const ViewParams& v, unsigned long long* keys, cudaStream_t s,
                           const Device& d) {
  constexpr auto k = k_render_basic<V, kUnroll, P>;
  k<<<geometry_grid<k, kUnroll>(n, d), kThreads, 0, s>>>(pts, n, v, keys);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_basic_p(int variant, const uint4* pts, uint32_t n, const ViewParams& v, unsigned long long* keys,
                           cudaStream_t s, const Device& d) {
  switch (variant) {
    case PCR_VARIANT_ATOMICMIN: return launch_basic_v<PCR_VARIANT_ATOMICMIN, P>(pts, n, v, keys, s, d);
    case PCR_VARIANT_EARLYZ: return launch_basic_v<PCR_VARIANT_EARLYZ, P>(pts, n, v, keys, s, d);
    case PCR_VARIANT_DEDUP: return launch_basic_v<PCR_VARIANT_DEDUP, P>(pts, n, v, keys, s, d);
    case PCR_VARIANT_DEDUP_EARLYZ: return launch_basic_v<PCR_VARIANT_DEDUP_EARLYZ, P>(pts, n, v, keys, s, d);
    case PCR_VARIANT_REDUCE: return launch_basic_v<PCR_VARIANT_REDUCE, P>(pts, n, v, keys, s, d);
    case PCR_VARIANT_REDUCE_EARLYZ: return launch_basic_v<PCR_VARIANT_REDUCE_EARLYZ, P>(pts, n, v, keys, s, d);
    case PCR_VARIANT_JUST_SET: return launch_basic_v<PCR_VARIANT_JUST_SET, P>(pts, n, v, keys, s, d);
    default: return cudaErrorInvalidValue;
  }
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
  return launch_basic_p<kPayloadIndex>(variant, pts, n, v, keys, s, d);
}

cudaError_t launch_render_rgb(int variant, const uint4* pts, uint32_t n, const ViewParams& v,
                              unsigned long long* keys, cudaStream_t s, const Device& d) {
  if (n == 0) return cudaSuccess;
  return launch_basic_p<kPayloadRgb>(variant, pts, n, v, keys, s, d);
}

cudaError_t launch_render_busy(const uint4* pts, uint32_t n, const ViewParams& v, unsigned long long* keys,
                               uint32_t* locks, uint64_t limit_ns, cudaStream_t s, const Device& d) {
  if (n == 0) return cudaSuccess;
  constexpr auto k = k_render_busy<kUnroll>;
  k<<<geometry_grid<k, kUnroll>(n, d), kThreads, 0, s>>>(pts, n, v, keys, locks, limit_ns);
  return cudaGetLastError();
}

cudaError_t launch_fill_u32(uint32_t* p, uint64_t count, uint32_t value, cudaStream_t s, const Device& d) {
  if (count == 0) return cudaSuccess;
  k_fill_u32<<<screen_grid(count, d), kThreads, 0, s>>>(p, count, value);
  return cudaGetLastError();
}

cudaError_t launch_resolve_rgb(const unsigned long long* keys, uint64_t npx, uint32_t background, uint32_t* out,
                               cudaStream_t s, const Device& d) {
  if (npx == 0) return cudaSuccess;
  k_resolve_rgb<<<screen_grid(npx, d), kThreads, 0, s>>>(keys, npx, background, out);
  return cudaGetLastError();
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

template <bool AGG, bool V8>
void launch_color_k(const uint4* pts, uint32_t n, const ViewParams& v, float depth_factor, const uint32_t* depth,
                    unsigned long long* rg, unsigned long long* ba, cudaStream_t s, const Device& d) {
  constexpr auto k = k_hq_color<AGG, kUnroll, V8>;
  k<<<geometry_grid<k, kUnroll>(n, d), kThreads, 0, s>>>(pts, n, v, depth_factor, depth, rg, ba);
}

cudaError_t launch_hq_color(int variant, const uint4* pts, uint32_t n, const ViewParams& v, float depth_factor,
                            const uint32_t* depth, unsigned long long* rg, unsigned long long* ba, cudaStream_t s,
                            const Device& d) {
  if (n == 0) return cudaSuccess;
  // every variant but the basic one groups colours before adding
  const bool agg = variant != PCR_VARIANT_ATOMICMIN;
  if (!agg) launch_color_k<false, false>(pts, n, v, depth_factor, depth, rg, ba, s, d);
  else if (pairs_aligned(pts)) launch_color_k<true, kCanPairLoad>(pts, n, v, depth_factor, depth, rg, ba, s, d);
  else launch_color_k<true, false>(pts, n, v, depth_factor, depth, rg, ba, s, d);
  return cudaGetLastError();
}

template <int P>
void prewarm_basic(const Device& d) {
  geometry_grid<k_render_basic<PCR_VARIANT_ATOMICMIN, kUnroll, P>, kUnroll>(1, d);
  geometry_grid<k_render_basic<PCR_VARIANT_EARLYZ, kUnroll, P>, kUnroll>(1, d);
  geometry_grid<k_render_basic<PCR_VARIANT_DEDUP, kUnroll, P>, kUnroll>(1, d);
  geometry_grid<k_render_basic<PCR_VARIANT_DEDUP_EARLYZ, kUnroll, P>, kUnroll>(1, d);
  geometry_grid<k_render_basic<PCR_VARIANT_REDUCE, kUnroll, P>, kUnroll>(1, d);
  geometry_grid<k_render_basic<PCR_VARIANT_REDUCE_EARLYZ, kUnroll, P>, kUnroll>(1, d);
  geometry_grid<k_render_basic<PCR_VARIANT_JUST_SET, kUnroll, P>, kUnroll>(1, d);
}

// Every single-view geometry kernel's occupancy query (cached per kernel):
// run once before a stream capture records launches.
void prewarm_single_view(const Device& d) {
  prewarm_basic<kPayloadIndex>(d);
  prewarm_basic<kPayloadRgb>(d);
  geometry_grid<k_render_busy<kUnroll>, kUnroll>(1, d);
  geometry_grid<k_hq_depth<PCR_VARIANT_ATOMICMIN, kUnroll>, kUnroll>(1, d);
  geometry_grid<k_hq_depth<PCR_VARIANT_EARLYZ, kUnroll>, kUnroll>(1, d);
  geometry_grid<k_hq_depth<PCR_VARIANT_DEDUP, kUnroll>, kUnroll>(1, d);
  geometry_grid<k_hq_depth<PCR_VARIANT_DEDUP_EARLYZ, kUnroll>, kUnroll>(1, d);
  geometry_grid<k_hq_color<false, kUnroll, false>, kUnroll>(1, d);
  geometry_grid<k_hq_color<true, kUnroll, kCanPairLoad>, kUnroll>(1, d);
  geometry_grid<k_hq_color<true, kUnroll, false>, kUnroll>(1, d);
  geometry_grid<k_hq1r_color<false, kUnroll, false>, kUnroll>(1, d);
  geometry_grid<k_hq1r_color<true, kUnroll, kCanPairLoad>, kUnroll>(1, d);
  geometry_grid<k_hq1r_color<true, kUnroll, false>, kUnroll>(1, d);
}

template <bool AGG, bool V8>
void launch_hq1r_k(const uint4* pts, uint32_t n, const ViewParams& v, float depth_factor, const uint32_t* depth,
                   unsigned long long* primary, unsigned long long* rg, unsigned long long* ba, cudaStream_t s,
                   const Device& d) {
  constexpr auto k = k_hq1r_color<AGG, kUnroll, V8>;
  k<<<geometry_grid<k, kUnroll>(n, d), kThreads, 0, s>>>(pts, n, v, depth_factor, depth, primary, rg, ba);
}

cudaError_t launch_hq1r_color(int variant, const uint4* pts, uint32_t n, const ViewParams& v, float depth_factor,
                              const uint32_t* depth, unsigned long long* primary, unsigned long long* rg,
                              unsigned long long* ba, cudaStream_t s, const Device& d) {
  if (n == 0) return cudaSuccess;
  const bool agg = variant != PCR_VARIANT_ATOMICMIN;
  if (!agg) launch_hq1r_k<false, false>(pts, n, v, depth_factor, depth, primary, rg, ba, s, d);
  else if (pairs_aligned(pts)) launch_hq1r_k<true, kCanPairLoad>(pts, n, v, depth_factor, depth, primary, rg, ba, s, d);
  else launch_hq1r_k<true, false>(pts, n, v, depth_factor, depth, primary, rg, ba, s, d);
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

cudaError_t read_and_clear_debug_counts(uint64_t out[4], cudaStream_t s, bool* available) {
#ifdef PCR_DEBUG
  *available = true;
  unsigned long long got[4];
  const unsigned long long zero[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemcpyFromSymbolAsync(got, g_debug_counts, sizeof(got), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_debug_counts, zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (int k = 0; k < 4; ++k) out[k] = got[k];
  return e;
#else
  (void)out;
  (void)s;
  *available = false;
  return cudaSuccess;
#endif
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
