// Batched rendering: many (cloud, view, resolution) jobs in one launch
// sequence (clear, geometry phase 1, geometry phase 2, resolve), capturable
// as one CUDA graph.
//
// Each pass over a cloud's points projects every point for a group of that
// cloud's views.  Phase 1 (index 0 in the tables) writes the basic key (Sec.
// 3.1-3.2, with the early depth test) and the high-quality depth (Sec. 3.5)
// from one projection; phase 2 (index 1), after all depth buffers are
// complete, adds the high-quality colours (summed inside the warp first).  A
// group holds as many views as fit an L2 budget (framebuffer bytes the pass
// touches), packed first-fit by decreasing size, so the atomics and early
// depth reads of a pass stay in L2 while the point stream passes through; a
// view alone in its pass goes through the single-view kernels instead.  The
// passes of a phase are laid out as one sequence of 128-point slots (each
// pass padded to a multiple of 128) that a persistent grid walks in uniform
// chunks: clouds of uneven size need no work queue and nothing waits.
// Results equal the per-view calls bit for bit: minima and integer sums do
// not depend on order.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/pcr.h"
#include "common.cuh"
#include "geometry.cuh"
#include "launch.h"

namespace pcr {

namespace {

using namespace geom;

constexpr int kThreads = 256;
constexpr uint64_t kSlot = 128;  // cloud padding and the largest chunk (32 lanes x 4)


struct Tables {
  BatchHeader hdr;
  BatchCloud clouds[kBatchMaxClouds];
  BatchView views[kBatchMaxViews];
  BatchGroup groups[2][kBatchMaxViews];
  uint16_t order[2][kBatchMaxViews];
  // Per phase (0: keys and depth, 1: colours), the views that are alone in
  // their pass (in phase 0 only those with one frame) and run through the
  // single-view kernels instead; the host reads these from its copy of the
  // tables when it launches the batch.
  uint32_t num_single[2];
  uint16_t single[2][kBatchMaxViews];
};

// The kernels copy the tables they read into dynamic shared memory, sized
// to the batch: header, clouds, views and (geometry phases) the phase's
// groups and view order, each 16-byte aligned.  A batch of 64 views over a
// few clouds takes about 10 KB, so shared memory does not bound the resident
// blocks (the full 256 x 256 tables take 42 KB, under the 48 KB a launch
// gets without opting in).
struct SharedLayout {
  uint32_t clouds, views, groups, order, bytes;
};

__host__ __device__ constexpr uint32_t align16(uint32_t v) { return (v + 15u) & ~15u; }

__host__ __device__ inline SharedLayout shared_layout(uint32_t num_clouds, uint32_t num_views, uint32_t num_groups,
                                                      bool geometry) {
  SharedLayout l{};
  l.clouds = align16(sizeof(BatchHeader));
  l.views = l.clouds + align16(num_clouds * static_cast<uint32_t>(sizeof(BatchCloud)));
  l.groups = l.views + align16(num_views * static_cast<uint32_t>(sizeof(BatchView)));
  l.order = l.groups + (geometry ? align16(num_groups * static_cast<uint32_t>(sizeof(BatchGroup))) : 0u);
  l.bytes = l.order + (geometry ? align16(num_views * static_cast<uint32_t>(sizeof(uint16_t))) : 0u);
  return l;
}

// Views of the tables in shared memory.
struct Shared {
  const BatchHeader& hdr;
  const BatchCloud* clouds;
  const BatchView* views;
  const BatchGroup* groups;
  const uint16_t* order;
};

extern __shared__ __align__(16) unsigned char g_smem_tables[];

constexpr uint64_t align256(uint64_t v) { return (v + 255) & ~uint64_t(255); }

// Debug builds (PCR_DEBUG) check every visible slot's pixel against its
// view before any access; a failure sets PCR_DEVICE_ERROR_BOUNDS in this
// file's error word (read by pcr_last_device_error) and drops the slot.
#ifdef PCR_DEBUG
__device__ uint32_t g_batch_error_word;
#endif
template <int U>
__device__ __forceinline__ void debug_check_view_pixels(const ViewParams& vp, const uint32_t (&pix)[U],
                                                        bool (&vis)[U]) {
#ifdef PCR_DEBUG
  const uint64_t npx = static_cast<uint64_t>(vp.width) * vp.height;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (vis[u] && pix[u] >= npx) {
      atomicOr(&g_batch_error_word, static_cast<uint32_t>(PCR_DEVICE_ERROR_BOUNDS));
      vis[u] = false;
    }
  }
#else
  (void)vp;
  (void)pix;
  (void)vis;
#endif
}

// Copy the header, clouds, views and (phase >= 0) that phase's groups and
// order into shared memory.
__device__ __forceinline__ Shared load_tables(const Tables* __restrict__ g, int phase) {
  BatchHeader* hdr = reinterpret_cast<BatchHeader*>(g_smem_tables);
  if (threadIdx.x == 0) *hdr = g->hdr;
  __syncthreads();
  const SharedLayout l =
      shared_layout(hdr->num_clouds, hdr->num_views, phase >= 0 ? hdr->num_groups[phase] : 0u, phase >= 0);
  auto copy = [](const void* src, void* dst, uint32_t bytes) {
    const uint32_t* s4 = static_cast<const uint32_t*>(src);
    uint32_t* d4 = static_cast<uint32_t*>(dst);
    for (uint32_t i = threadIdx.x; i < bytes / 4; i += blockDim.x) d4[i] = s4[i];
  };
  copy(g->clouds, g_smem_tables + l.clouds, hdr->num_clouds * sizeof(BatchCloud));
  copy(g->views, g_smem_tables + l.views, hdr->num_views * sizeof(BatchView));
  if (phase >= 0) {
    copy(g->groups[phase], g_smem_tables + l.groups, hdr->num_groups[phase] * sizeof(BatchGroup));
    copy(g->order[phase], g_smem_tables + l.order, (hdr->num_views * sizeof(uint16_t) + 3) / 4 * 4);
  }
  __syncthreads();
  return Shared{*hdr, reinterpret_cast<const BatchCloud*>(g_smem_tables + l.clouds),
                reinterpret_cast<const BatchView*>(g_smem_tables + l.views),
                reinterpret_cast<const BatchGroup*>(g_smem_tables + l.groups),
                reinterpret_cast<const uint16_t*>(g_smem_tables + l.order)};
}

// Largest i in [0, count) with key(i) <= x (key(0) is 0, so i exists).
template <class Key>
__device__ __forceinline__ uint32_t last_not_above(uint32_t count, uint64_t x, Key key) {
  uint32_t lo = 0, hi = count;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) / 2;
    if (key(mid) <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// Walk the chunks (32 * U points) of every pass of a phase; f(group, r,
// base, ok) for each chunk of this warp.  Slot u of lane l holds point
// slot_index<U, L>(base, u) of the group's cloud (the layouts of the
// single-view kernels); in the consecutive layout, whole chunks of a 32-byte
// aligned cloud load their records in 32-byte pairs.
template <int U, int L, class F>
__device__ __forceinline__ void for_each_batch_chunk(const Shared& sh, int phase, uint64_t pol, F&& f) {
  static_assert(L == kInterleaved || U % 2 == 0, "records load in pairs");
  constexpr uint32_t kLaneStep = L == kConsecutive ? U : 1;
  const uint64_t warps_per_block = blockDim.x >> 5;
  const uint64_t warp = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  const uint64_t nwarps = gridDim.x * warps_per_block;
  constexpr uint64_t kChunk = 32ull * U;
  const uint64_t nchunks = sh.hdr.total_slots[phase] / kChunk;
  const uint32_t lane = lane_id();
  for (uint64_t g = warp; g < nchunks; g += nwarps) {
    const uint64_t slot0 = g * kChunk;
    const uint32_t gi =
        last_not_above(sh.hdr.num_groups[phase], slot0, [&](uint32_t i) { return sh.groups[i].first_slot; });
    const BatchGroup& grp = sh.groups[gi];
    const BatchCloud& cl = sh.clouds[grp.cloud];
    const uint64_t start = slot0 - grp.first_slot;
    const uint32_t base = static_cast<uint32_t>(start) + kLaneStep * lane;
    uint4 r[U];
    bool ok[U];
    if (L == kConsecutive && start + kChunk <= cl.n && (reinterpret_cast<uintptr_t>(cl.pts) & 31u) == 0) {
#pragma unroll
      for (int u = 0; u < U; u += 2) load_pair_stream(cl.pts + base + u, pol, r[u], r[u + 1]);
#pragma unroll
      for (int u = 0; u < U; ++u) ok[u] = true;
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint64_t i = slot_index<U, L>(base, u);
        ok[u] = i < cl.n;
        r[u] = ok[u] ? load_point_stream(cl.pts + i, pol) : make_uint4(0u, 0u, 0u, 0u);
      }
    }
    f(grp, r, base, ok);
  }
}

template <int U>
__device__ __forceinline__ void project_all(const ViewParams& vp, const uint4 (&r)[U], const bool (&ok)[U],
                                            uint32_t (&pix)[U], float (&w)[U], bool (&vis)[U]) {
  // project every slot (a slot past the cloud holds zeros), then mask: no
  // branch per slot, so the slots' work interleaves
  project_slots<U>(vp, r, pix, w, vis);
#pragma unroll
  for (int u = 0; u < U; ++u) vis[u] = vis[u] && ok[u];
  debug_check_view_pixels<U>(vp, pix, vis);
}

// Phase 1: per view of the pass, basic key and HQ depth, each with the
// early depth test (on GB300 the fastest exact form once the buffer is
// filling: warp deduplication saves no atomics after the early test), both
// from one projection.
template <int U, int T>
__global__ void __launch_bounds__(T) k_batch_phase1(const Tables* __restrict__ tables) {
  const Shared sh = load_tables(tables, 0);
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_fb = policy_evict_last();
  for_each_batch_chunk<U, kInterleaved>(sh, 0, pol_stream, [&](const BatchGroup& grp, const uint4(&r)[U], uint32_t base,
                                                 const bool(&ok)[U]) {
    for (uint32_t i = grp.first; i < grp.first + grp.count; ++i) {
      const BatchView& bv = sh.views[sh.order[i]];
      uint32_t pix[U];
      float w[U];
      bool vis[U];
      project_all<U>(bv.vp, r, ok, pix, w, vis);
      // both early reads of every slot first: one L2 round trip per view
      const bool basic = bv.flags & PCR_BATCH_BASIC;
      const bool hq = bv.flags & PCR_BATCH_HQ;
      unsigned long long seen_key[U];
      uint32_t seen_depth[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        seen_key[u] = (basic && vis[u]) ? load_relaxed_u64(bv.keys + pix[u]) : 0ull;
        seen_depth[u] = (hq && vis[u]) ? load_relaxed_u32(bv.depth + pix[u]) : 0u;
      }
      if (basic) {
#pragma unroll
        for (int u = 0; u < U; ++u)
          emit_key<PCR_VARIANT_EARLYZ>(bv.keys, vis[u], pix[u], make_key(w[u], slot_index<U, kInterleaved>(base, u)), seen_key[u], pol_fb);
      }
      if (hq) {
#pragma unroll
        for (int u = 0; u < U; ++u)
          emit_depth<PCR_VARIANT_EARLYZ>(bv.depth, vis[u], pix[u], __float_as_uint(w[u]), seen_depth[u],
                                               pol_fb);
      }
    }
  });
}

// Phase 2: HQ colours (warp-aggregated adds) for the HQ views of the pass.
// Held to 64 registers (1024 threads per SM) at either block size.
template <int U, int T>
__global__ void __launch_bounds__(T, 1024 / T) k_batch_phase2(const Tables* __restrict__ tables) {
  const Shared sh = load_tables(tables, 1);
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_fb = policy_evict_last();
  const float factor = sh.hdr.depth_factor;
  for_each_batch_chunk<U, kConsecutive>(sh, 1, pol_stream, [&](const BatchGroup& grp, const uint4(&r)[U], uint32_t,
                                                 const bool(&ok)[U]) {
    for (uint32_t i = grp.first; i < grp.first + grp.count; ++i) {
      const BatchView& bv = sh.views[sh.order[i]];
      uint32_t pix[U];
      float w[U];
      bool vis[U];
      project_all<U>(bv.vp, r, ok, pix, w, vis);
      bool contrib[U];
      contributes<U>(bv.depth, factor, pix, w, vis, contrib);
      emit_colors<U, true>(bv.rg, bv.ba, contrib, pix, r, pol_fb);
    }
  });
}

// Clear and resolve walk the pixels of all views as one sequence.  The view
// of a pixel is found by one search per warp (lane 0's pixel); lanes whose
// pixel lies past that view's end search on their own.
__device__ __forceinline__ uint32_t view_of_pixel(const Shared& sh, uint64_t p) {
  const uint64_t p0 = __shfl_sync(kFullMask, p, 0);
  uint32_t vi = 0;
  if (lane_id() == 0)
    vi = last_not_above(sh.hdr.num_views, p0, [&](uint32_t i) { return sh.views[i].first_pixel; });
  vi = __shfl_sync(kFullMask, vi, 0);
  const uint64_t end = vi + 1 < sh.hdr.num_views ? sh.views[vi + 1].first_pixel : sh.hdr.total_pixels;
  if (p >= end) vi = last_not_above(sh.hdr.num_views, p, [&](uint32_t i) { return sh.views[i].first_pixel; });
  return vi;
}

__global__ void __launch_bounds__(kThreads) k_batch_clear(const Tables* __restrict__ tables) {
  const Shared sh = load_tables(tables, -1);
  const BatchHeader& hdr = sh.hdr;
  const BatchView* views = sh.views;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  const uint64_t rounds = (hdr.total_pixels + stride - 1) / stride;  // every lane runs the same rounds
  for (uint64_t k = 0; k < rounds; ++k) {
    const uint64_t p = k * stride + blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
    const uint32_t vi = view_of_pixel(sh, p < hdr.total_pixels ? p : hdr.total_pixels - 1);
    if (p >= hdr.total_pixels) continue;
    const BatchView& bv = views[vi];
    const uint64_t q = p - bv.first_pixel;
    if (bv.flags & PCR_BATCH_BASIC) bv.keys[q] = kEmptyKey;
    if (bv.flags & PCR_BATCH_HQ) {
      bv.depth[q] = kInfBits;
      bv.rg[q] = 0ull;
      bv.ba[q] = 0ull;
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_batch_resolve(const Tables* __restrict__ tables) {
  const Shared sh = load_tables(tables, -1);
  const BatchHeader& hdr = sh.hdr;
  const BatchView* views = sh.views;
  const BatchCloud* clouds = sh.clouds;
  const uint32_t background = hdr.background;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  const uint64_t rounds = (hdr.total_pixels + stride - 1) / stride;  // every lane runs the same rounds
  for (uint64_t k = 0; k < rounds; ++k) {
    const uint64_t p = k * stride + blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
    const uint32_t vi = view_of_pixel(sh, p < hdr.total_pixels ? p : hdr.total_pixels - 1);
    if (p >= hdr.total_pixels) continue;
    const BatchView& bv = views[vi];
    const uint64_t q = p - bv.first_pixel;
    if ((bv.flags & PCR_BATCH_BASIC) && bv.image) {
      const unsigned long long k = bv.keys[q];
      const uint32_t idx = static_cast<uint32_t>(k);
      const BatchCloud& cl = clouds[bv.cloud];
      uint32_t c = background;
      if (k != kEmptyKey && idx < cl.n) c = __ldg(reinterpret_cast<const uint32_t*>(cl.pts) + 4ull * idx + 3);
      bv.image[q] = c;
    }
    if ((bv.flags & PCR_BATCH_HQ) && bv.hq_image) {
      const unsigned long long s_rg = bv.rg[q];
      const unsigned long long s_ba = bv.ba[q];
      const uint32_t a = static_cast<uint32_t>(s_ba);
      uint32_t c = background;
      if (a != 0) {
        c = min(static_cast<uint32_t>(s_rg >> 32) / a, 255u) | (min(static_cast<uint32_t>(s_rg) / a, 255u) << 8) |
            (min(static_cast<uint32_t>(s_ba >> 32) / a, 255u) << 16) | 0xFF000000u;
      }
      bv.hq_image[q] = c;
    }
  }
}

// Launch configurations the autotuner chooses among: threads per block, and
// points per lane of the two geometry phases (phase 2 keeps more state per
// point), and where the colours are added.  Configuration c: threads
// 256 << ((c >> 2) & 1), phase-1 points per lane (c & 2) ? 2 : 4, phase-2
// (c & 1) ? 2 : 4; with c & 8, every HQ view's colours are added by the
// single-view colour pass (one pass over the points per view, the kernel
// with the fewest instructions per point) and phase 2 is not launched.
// Configuration 0 is the default.
constexpr int kNumConfigs = 16;

// Resident blocks per SM of a geometry kernel with `smem` bytes of tables
// (the occupancy query is host arithmetic; its first call per kernel loads
// the kernel, which the prewarm does before any capture).
template <auto K>
int batch_resident(int threads, uint32_t smem) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, K, threads, smem) != cudaSuccess || b < 1) b = 1;
  return b;
}

template <auto K, int T>
void launch_persistent(const Tables* t, uint32_t smem, cudaStream_t s, const Device& d) {
  K<<<d.num_sms * batch_resident<K>(T, smem), T, smem, s>>>(t);
}

template <int T>
void launch_phase(const Tables* t, uint32_t smem, int config, int phase, cudaStream_t s, const Device& d) {
  if (phase == 0) {
    if (config & 2) launch_persistent<k_batch_phase1<2, T>, T>(t, smem, s, d);
    else launch_persistent<k_batch_phase1<4, T>, T>(t, smem, s, d);
  } else {
    if (config & 1) launch_persistent<k_batch_phase2<2, T>, T>(t, smem, s, d);
    else launch_persistent<k_batch_phase2<4, T>, T>(t, smem, s, d);
  }
}

void launch_batch_phase(const Tables& h, const Tables* t, int config, int phase, cudaStream_t s, const Device& d) {
  const uint32_t smem = shared_layout(h.hdr.num_clouds, h.hdr.num_views, h.hdr.num_groups[phase], true).bytes;
  if (config & 4) launch_phase<512>(t, smem, config, phase, s, d);
  else launch_phase<256>(t, smem, config, phase, s, d);
}

// The single-view kernels of one view and phase (index): 0 the basic keys
// (early-z) and the HQ depth (dedup+early-z), 1 the HQ colours (warp
// aggregated) -- the kernels pcr_render_basic and pcr_render_hq run.
cudaError_t launch_single(const Tables& h, uint32_t vi, int phase, cudaStream_t s, const Device& d) {
  const BatchView& v = h.views[vi];
  const BatchCloud& c = h.clouds[v.cloud];
  cudaError_t e = cudaSuccess;
  if (phase == 0) {
    if (v.flags & PCR_BATCH_BASIC) e = launch_render_basic(PCR_VARIANT_EARLYZ, c.pts, c.n, v.vp, v.keys, s, d);
    if (e == cudaSuccess && (v.flags & PCR_BATCH_HQ))
      e = launch_hq_depth(PCR_VARIANT_DEDUP_EARLYZ, c.pts, c.n, v.vp, v.depth, s, d);
  } else if (v.flags & PCR_BATCH_HQ) {
    e = launch_hq_color(PCR_VARIANT_DEDUP_EARLYZ, c.pts, c.n, v.vp, h.hdr.depth_factor, v.depth, v.rg, v.ba, s, d);
  }
  return e;
}

template <int T>
void prewarm_phases() {
  batch_resident<k_batch_phase1<4, T>>(T, 0);
  batch_resident<k_batch_phase2<4, T>>(T, 0);
  batch_resident<k_batch_phase1<2, T>>(T, 0);
  batch_resident<k_batch_phase2<2, T>>(T, 0);
}

}  // namespace

uint64_t batch_workspace_bytes() { return align256(sizeof(Tables)); }

int batch_num_configs() { return kNumConfigs; }

namespace {

// Pack the views of each cloud that take part in a phase into passes whose
// framebuffer bytes fit the L2 budget (first fit, largest first); a view
// larger than the budget gets a pass of its own.  A pass of one view shares
// no point loads: that view goes to the phase's single-view list instead (in
// the keys-and-depth phase, index 0, only when it asks for one frame; with
// both, the batch pass still reads its points once for the two).
void build_groups(Tables* t, const pcr_batch_cloud* clouds, uint32_t num_clouds, const pcr_batch_view* views,
                  uint32_t num_views, int phase, uint64_t l2_budget) {
  uint32_t ng = 0, nord = 0, nsingle = 0;
  uint64_t slot = 0;
  for (uint32_t c = 0; c < num_clouds; ++c) {
    std::vector<std::pair<uint64_t, uint32_t>> mine;  // (bytes, view)
    for (uint32_t i = 0; i < num_views; ++i) {
      const pcr_batch_view& v = views[i];
      if (v.cloud != c) continue;
      const uint64_t px = static_cast<uint64_t>(v.width) * static_cast<uint64_t>(v.height);
      uint64_t bytes = 0;
      if (phase == 0) bytes = px * (((v.flags & PCR_BATCH_BASIC) ? 8u : 0u) + ((v.flags & PCR_BATCH_HQ) ? 4u : 0u));
      else if (v.flags & PCR_BATCH_HQ) bytes = px * 20u;  // depth read, two 64-bit sums
      if (bytes > 0) mine.emplace_back(bytes, i);
    }
    std::stable_sort(mine.begin(), mine.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    std::vector<std::vector<uint32_t>> bins;
    std::vector<uint64_t> used;
    for (const auto& [bytes, vi] : mine) {
      size_t b = 0;
      while (b < bins.size() && used[b] + bytes > l2_budget) ++b;
      if (b == bins.size()) {
        bins.emplace_back();
        used.push_back(0);
      }
      bins[b].push_back(vi);
      used[b] += bytes;
    }
    const uint64_t padded = (clouds[c].n + kSlot - 1) / kSlot * kSlot;
    for (const auto& bin : bins) {
      const uint32_t f = views[bin[0]].flags;
      if (bin.size() == 1 && (phase == 1 || f != (PCR_BATCH_BASIC | PCR_BATCH_HQ))) {
        t->single[phase][nsingle++] = static_cast<uint16_t>(bin[0]);
        continue;
      }
      BatchGroup& g = t->groups[phase][ng++];
      g.cloud = c;
      g.first = nord;
      g.count = static_cast<uint32_t>(bin.size());
      g.first_slot = slot;
      slot += padded;
      for (uint32_t vi : bin) t->order[phase][nord++] = static_cast<uint16_t>(vi);
    }
  }
  t->hdr.num_groups[phase] = ng;
  t->hdr.total_slots[phase] = slot;
  t->num_single[phase] = nsingle;
}

}  // namespace

uint64_t batch_tables_bytes() { return sizeof(Tables); }

void batch_build_tables(const pcr_batch_cloud* clouds, uint32_t num_clouds, const pcr_batch_view* views,
                        uint32_t num_views, float depth_factor, uint32_t background, void* host_tables,
                        uint64_t l2_budget) {
  Tables* t = new (host_tables) Tables();
  t->hdr.num_clouds = num_clouds;
  t->hdr.num_views = num_views;
  t->hdr.depth_factor = depth_factor;
  t->hdr.background = background;
  for (uint32_t c = 0; c < num_clouds; ++c) {
    t->clouds[c].pts = static_cast<const uint4*>(clouds[c].points);
    t->clouds[c].n = static_cast<uint32_t>(clouds[c].n);
  }
  uint64_t pixel = 0;
  uint32_t hq = 0;
  for (uint32_t j = 0; j < num_views; ++j) {
    const pcr_batch_view& in = views[j];
    BatchView& bv = t->views[j];
    for (int k = 0; k < 4; ++k) {
      bv.vp.r0[k] = in.matrix[k];
      bv.vp.r1[k] = in.matrix[4 + k];
      bv.vp.r3[k] = in.matrix[12 + k];
    }
    bv.vp.fw = static_cast<float>(in.width);
    bv.vp.fh = static_cast<float>(in.height);
    bv.vp.width = static_cast<uint32_t>(in.width);
    bv.vp.height = static_cast<uint32_t>(in.height);
    bv.cloud = in.cloud;
    bv.flags = in.flags;
    bv.keys = static_cast<unsigned long long*>(in.keys);
    bv.image = static_cast<uint32_t*>(in.image);
    bv.depth = static_cast<uint32_t*>(in.hq_depth);
    bv.rg = static_cast<unsigned long long*>(in.hq_rg);
    bv.ba = static_cast<unsigned long long*>(in.hq_ba);
    bv.hq_image = static_cast<uint32_t*>(in.hq_image);
    bv.first_pixel = pixel;
    pixel += static_cast<uint64_t>(in.width) * static_cast<uint64_t>(in.height);
    if (in.flags & PCR_BATCH_HQ) ++hq;
  }
  t->hdr.total_pixels = pixel;
  t->hdr.hq_views = hq;
  build_groups(t, clouds, num_clouds, views, num_views, 0, l2_budget);
  build_groups(t, clouds, num_clouds, views, num_views, 1, l2_budget);
}

cudaError_t batch_prepare(const pcr_batch_cloud* clouds, uint32_t num_clouds, const pcr_batch_view* views,
                          uint32_t num_views, float depth_factor, uint32_t background, void* host_tables,
                          void* workspace, cudaStream_t s, uint64_t l2_budget) {
  batch_build_tables(clouds, num_clouds, views, num_views, depth_factor, background, host_tables, l2_budget);
  cudaError_t e = cudaMemcpyAsync(workspace, host_tables, sizeof(Tables), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

cudaError_t batch_prewarm(const Device& d) {
  prewarm_phases<256>();
  prewarm_phases<512>();
  prewarm_single_view(d);
  return cudaGetLastError();
}

cudaError_t read_and_clear_batch_error_word(uint32_t* out, cudaStream_t s) {
  *out = 0;
#ifdef PCR_DEBUG
  const uint32_t zero = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_batch_error_word, sizeof(uint32_t), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_batch_error_word, &zero, sizeof(uint32_t), 0,
                                                    cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
#else
  (void)s;
  return cudaSuccess;
#endif
}

int batch_launch_count(const void* host_tables, int config) {
  const Tables& h = *static_cast<const Tables*>(host_tables);
  auto single = [&](uint32_t vi, int phase) {
    const BatchView& v = h.views[vi];
    if (h.clouds[v.cloud].n == 0) return 0;
    if (phase == 1) return (v.flags & PCR_BATCH_HQ) ? 1 : 0;
    return ((v.flags & PCR_BATCH_BASIC) ? 1 : 0) + ((v.flags & PCR_BATCH_HQ) ? 1 : 0);
  };
  int count = 2 + (h.hdr.total_slots[0] > 0 ? 1 : 0);
  for (uint32_t k = 0; k < h.num_single[0]; ++k) count += single(h.single[0][k], 0);
  if (batch_config_single_colors(config)) {
    for (uint32_t vi = 0; vi < h.hdr.num_views; ++vi) count += single(vi, 1);
  } else {
    count += h.hdr.total_slots[1] > 0 ? 1 : 0;
    for (uint32_t k = 0; k < h.num_single[1]; ++k) count += single(h.single[1][k], 1);
  }
  return count;
}

int batch_config_threads(int config) { return 256 << ((config >> 2) & 1); }
int batch_config_unroll(int config, int phase) { return (config & (phase == 0 ? 2 : 1)) ? 2 : 4; }
bool batch_config_single_colors(int config) { return (config & 8) != 0; }

// clear, phase 1 (the batch passes, then the single-view passes of views
// alone in theirs), phase 2 (likewise, or every HQ view single-view), and
// resolve, in stream order: phase 2 reads complete depth buffers.
cudaError_t batch_launch(const void* host_tables, const void* workspace, int config, cudaStream_t s,
                         const Device& d) {
  if (config < 0 || config >= kNumConfigs) return cudaErrorInvalidValue;
  const Tables& h = *static_cast<const Tables*>(host_tables);
  const Tables* t = static_cast<const Tables*>(workspace);
  const int screen_blocks = d.num_sms * 8;
  const uint32_t screen_smem = shared_layout(h.hdr.num_clouds, h.hdr.num_views, 0, false).bytes;
  k_batch_clear<<<screen_blocks, kThreads, screen_smem, s>>>(t);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && h.hdr.total_slots[0] > 0) {
    launch_batch_phase(h, t, config, 0, s, d);
    e = cudaGetLastError();
  }
  for (uint32_t k = 0; k < h.num_single[0] && e == cudaSuccess; ++k) e = launch_single(h, h.single[0][k], 0, s, d);
  if (batch_config_single_colors(config)) {
    for (uint32_t vi = 0; vi < h.hdr.num_views && e == cudaSuccess; ++vi) e = launch_single(h, vi, 1, s, d);
  } else {
    if (e == cudaSuccess && h.hdr.total_slots[1] > 0) {
      launch_batch_phase(h, t, config, 1, s, d);
      e = cudaGetLastError();
    }
    for (uint32_t k = 0; k < h.num_single[1] && e == cudaSuccess; ++k) e = launch_single(h, h.single[1][k], 1, s, d);
  }
  if (e != cudaSuccess) return e;
  k_batch_resolve<<<screen_blocks, kThreads, screen_smem, s>>>(t);
  return cudaGetLastError();
}

}  // namespace pcr
