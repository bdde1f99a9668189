// Batched rendering: many (cloud, view, resolution) jobs in one launch
// sequence (clear, geometry phase 1, geometry phase 2, resolve), capturable
// as one CUDA graph.
//
// Each cloud's points are read once per phase and projected for every view
// of that cloud.  Phase 1 writes the basic key (Sec. 3.1-3.4, warp
// deduplication plus early depth test) and the high-quality depth (Sec. 3.5)
// from one projection; phase 2, after the depth buffers are complete, adds
// the high-quality colours.  A frame of V views of a cloud thus reads its
// points twice instead of 3V times.  Clouds of uneven size are laid out as
// one sequence of 128-point slots (each cloud padded to a multiple of 128),
// which a persistent grid walks in uniform chunks, so no work queue and no
// waiting is needed.  Results equal the per-view calls bit for bit: minima
// and integer sums do not depend on order.
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
};

constexpr uint64_t align256(uint64_t v) { return (v + 255) & ~uint64_t(255); }

__device__ __forceinline__ void load_tables(const Tables* __restrict__ g, BatchHeader& hdr, BatchCloud* clouds,
                                            BatchView* views) {
  if (threadIdx.x == 0) hdr = g->hdr;
  __syncthreads();
  const uint32_t nc = hdr.num_clouds, nv = hdr.num_views;
  const uint32_t* src = reinterpret_cast<const uint32_t*>(g->clouds);
  uint32_t* dst = reinterpret_cast<uint32_t*>(clouds);
  for (uint32_t i = threadIdx.x; i < nc * (sizeof(BatchCloud) / 4); i += blockDim.x) dst[i] = src[i];
  src = reinterpret_cast<const uint32_t*>(g->views);
  dst = reinterpret_cast<uint32_t*>(views);
  for (uint32_t i = threadIdx.x; i < nv * (sizeof(BatchView) / 4); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
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

// Walk the chunks (32 * U points) of all clouds; f(cloud, r, base, ok) for
// each chunk of this warp whose cloud passes `want` (others are not read).
template <int U, class W, class F>
__device__ __forceinline__ void for_each_batch_chunk(const BatchHeader& hdr, const BatchCloud* clouds, uint64_t pol,
                                                     W&& want, F&& f) {
  const uint64_t warps_per_block = blockDim.x >> 5;
  const uint64_t warp = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  const uint64_t nwarps = gridDim.x * warps_per_block;
  constexpr uint64_t kChunk = 32ull * U;
  const uint64_t nchunks = hdr.total_slots / kChunk;
  const uint32_t lane = lane_id();
  for (uint64_t g = warp; g < nchunks; g += nwarps) {
    const uint64_t slot0 = g * kChunk;
    const uint32_t c = last_not_above(hdr.num_clouds, slot0, [&](uint32_t i) { return clouds[i].first_slot; });
    const BatchCloud& cl = clouds[c];
    if (!want(cl)) continue;
    const uint32_t base = static_cast<uint32_t>(slot0 - cl.first_slot) + lane;
    uint4 r[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = static_cast<uint64_t>(base) + 32ull * u;
      ok[u] = i < cl.n;
      r[u] = ok[u] ? load_point_stream(cl.pts + i, pol) : make_uint4(0u, 0u, 0u, 0u);
    }
    f(c, r, base, ok);
  }
}

template <int U>
__device__ __forceinline__ void project_all(const ViewParams& vp, const uint4 (&r)[U], const bool (&ok)[U],
                                            uint32_t (&pix)[U], float (&w)[U], bool (&vis)[U]) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    pix[u] = 0;
    w[u] = 0.0f;
    vis[u] = ok[u] && project(vp, __uint_as_float(r[u].x), __uint_as_float(r[u].y), __uint_as_float(r[u].z), pix[u],
                              w[u]);
  }
}

// Phase 1: per view of the chunk's cloud, basic key (dedup + early-z) and
// HQ depth (dedup + early-z), both from one projection.
template <int U>
__global__ void __launch_bounds__(kThreads) k_batch_phase1(const Tables* __restrict__ tables) {
  __shared__ BatchHeader hdr;
  __shared__ BatchCloud clouds[kBatchMaxClouds];
  __shared__ BatchView views[kBatchMaxViews];
  load_tables(tables, hdr, clouds, views);
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_fb = policy_evict_last();
  auto any_view = [](const BatchCloud& cl) { return cl.num_views > 0; };
  for_each_batch_chunk<U>(hdr, clouds, pol_stream, any_view, [&](uint32_t c, const uint4(&r)[U], uint32_t base,
                                                                 const bool(&ok)[U]) {
    const BatchCloud& cl = clouds[c];
    for (uint32_t vi = cl.first_view; vi < cl.first_view + cl.num_views; ++vi) {
      const BatchView& bv = views[vi];
      uint32_t pix[U];
      float w[U];
      bool vis[U];
      project_all<U>(bv.vp, r, ok, pix, w, vis);
      if (bv.flags & PCR_BATCH_BASIC) {
        unsigned long long seen[U];
#pragma unroll
        for (int u = 0; u < U; ++u) seen[u] = vis[u] ? load_relaxed_u64(bv.keys + pix[u]) : 0ull;
#pragma unroll
        for (int u = 0; u < U; ++u)
          emit_key<PCR_VARIANT_DEDUP_EARLYZ>(bv.keys, vis[u], pix[u], w[u], base + 32u * u, seen[u], pol_fb);
      }
      if (bv.flags & PCR_BATCH_HQ) {
        uint32_t seen[U];
#pragma unroll
        for (int u = 0; u < U; ++u) seen[u] = vis[u] ? load_relaxed_u32(bv.depth + pix[u]) : 0u;
#pragma unroll
        for (int u = 0; u < U; ++u)
          emit_depth<PCR_VARIANT_DEDUP_EARLYZ>(bv.depth, vis[u], pix[u], __float_as_uint(w[u]), seen[u], pol_fb);
      }
    }
  });
}

// Phase 2: HQ colours (warp-aggregated adds) for every HQ view.
template <int U>
__global__ void __launch_bounds__(kThreads) k_batch_phase2(const Tables* __restrict__ tables) {
  __shared__ BatchHeader hdr;
  __shared__ BatchCloud clouds[kBatchMaxClouds];
  __shared__ BatchView views[kBatchMaxViews];
  load_tables(tables, hdr, clouds, views);
  if (hdr.hq_views == 0) return;
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_fb = policy_evict_last();
  const float factor = hdr.depth_factor;
  auto any_hq = [](const BatchCloud& cl) { return cl.hq_views > 0; };
  for_each_batch_chunk<U>(hdr, clouds, pol_stream, any_hq, [&](uint32_t c, const uint4(&r)[U], uint32_t,
                                                               const bool(&ok)[U]) {
    const BatchCloud& cl = clouds[c];
    for (uint32_t vi = cl.first_view; vi < cl.first_view + cl.num_views; ++vi) {
      const BatchView& bv = views[vi];
      if (!(bv.flags & PCR_BATCH_HQ)) continue;
      uint32_t pix[U];
      float w[U];
      bool vis[U];
      project_all<U>(bv.vp, r, ok, pix, w, vis);
      uint32_t d[U];
#pragma unroll
      for (int u = 0; u < U; ++u) d[u] = vis[u] ? __ldg(bv.depth + pix[u]) : 0u;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool contrib = vis[u] && w[u] <= __fmul_rn(__uint_as_float(d[u]), factor);
        emit_color<true>(bv.rg, bv.ba, contrib, pix[u], r[u].w, pol_fb);
      }
    }
  });
}

// Clear and resolve walk the pixels of all views as one sequence.
__global__ void __launch_bounds__(kThreads) k_batch_clear(const Tables* __restrict__ tables) {
  __shared__ BatchHeader hdr;
  __shared__ BatchCloud clouds[kBatchMaxClouds];
  __shared__ BatchView views[kBatchMaxViews];
  load_tables(tables, hdr, clouds, views);
  for (uint64_t p = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; p < hdr.total_pixels;
       p += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint32_t vi = last_not_above(hdr.num_views, p, [&](uint32_t i) { return views[i].first_pixel; });
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
  __shared__ BatchHeader hdr;
  __shared__ BatchCloud clouds[kBatchMaxClouds];
  __shared__ BatchView views[kBatchMaxViews];
  load_tables(tables, hdr, clouds, views);
  const uint32_t background = hdr.background;
  for (uint64_t p = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; p < hdr.total_pixels;
       p += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint32_t vi = last_not_above(hdr.num_views, p, [&](uint32_t i) { return views[i].first_pixel; });
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

// Launch configurations the autotuner chooses among: points per lane, and
// resident blocks per SM (0 = as many as fit).
struct BatchConfig {
  int unroll;
  int blocks_per_sm;
};
constexpr BatchConfig kConfigs[] = {{4, 0}, {2, 0}, {4, 2}, {2, 2}};
constexpr int kNumConfigs = sizeof(kConfigs) / sizeof(kConfigs[0]);

template <auto K>
int batch_resident() {
  static const int blocks = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, K, kThreads, 0) != cudaSuccess || b < 1) b = 1;
    return b;
  }();
  return blocks;
}

template <int U>
cudaError_t launch_phases(const Tables* t, int bps, cudaStream_t s, const Device& d) {
  constexpr auto p1 = k_batch_phase1<U>;
  constexpr auto p2 = k_batch_phase2<U>;
  const int b1 = bps > 0 ? std::min(bps, batch_resident<p1>()) : batch_resident<p1>();
  const int b2 = bps > 0 ? std::min(bps, batch_resident<p2>()) : batch_resident<p2>();
  p1<<<d.num_sms * b1, kThreads, 0, s>>>(t);
  p2<<<d.num_sms * b2, kThreads, 0, s>>>(t);
  return cudaGetLastError();
}

}  // namespace

uint64_t batch_workspace_bytes() { return align256(sizeof(Tables)); }

int batch_num_configs() { return kNumConfigs; }

cudaError_t batch_prepare(const pcr_batch_cloud* clouds, uint32_t num_clouds, const pcr_batch_view* views,
                          uint32_t num_views, float depth_factor, uint32_t background, void* workspace,
                          cudaStream_t s) {
  std::vector<uint32_t> order(num_views);
  for (uint32_t i = 0; i < num_views; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](uint32_t a, uint32_t b) { return views[a].cloud < views[b].cloud; });
  Tables* t = new (std::nothrow) Tables();
  if (!t) return cudaErrorMemoryAllocation;
  t->hdr.num_clouds = num_clouds;
  t->hdr.num_views = num_views;
  t->hdr.depth_factor = depth_factor;
  t->hdr.background = background;
  uint64_t slot = 0;
  for (uint32_t c = 0; c < num_clouds; ++c) {
    BatchCloud& bc = t->clouds[c];
    bc.pts = static_cast<const uint4*>(clouds[c].points);
    bc.n = static_cast<uint32_t>(clouds[c].n);
    bc.first_slot = slot;
    slot += (clouds[c].n + kSlot - 1) / kSlot * kSlot;
    bc.first_view = 0;
    bc.num_views = 0;
    bc.hq_views = 0;
  }
  t->hdr.total_slots = slot;
  uint64_t pixel = 0;
  uint32_t hq = 0;
  for (uint32_t j = 0; j < num_views; ++j) {
    const pcr_batch_view& in = views[order[j]];
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
    BatchCloud& bc = t->clouds[in.cloud];
    if (bc.num_views == 0) bc.first_view = j;
    ++bc.num_views;
    if (in.flags & PCR_BATCH_HQ) ++bc.hq_views;
  }
  t->hdr.total_pixels = pixel;
  t->hdr.hq_views = hq;
  cudaError_t e = cudaMemcpyAsync(workspace, t, sizeof(Tables), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  delete t;
  return e;
}

cudaError_t batch_prewarm(const Device&) {
  batch_resident<k_batch_phase1<4>>();
  batch_resident<k_batch_phase2<4>>();
  batch_resident<k_batch_phase1<2>>();
  batch_resident<k_batch_phase2<2>>();
  return cudaGetLastError();
}

cudaError_t batch_launch(const void* workspace, int config, cudaStream_t s, const Device& d) {
  if (config < 0 || config >= kNumConfigs) return cudaErrorInvalidValue;
  const Tables* t = static_cast<const Tables*>(workspace);
  const int screen_blocks = d.num_sms * 8;
  k_batch_clear<<<screen_blocks, kThreads, 0, s>>>(t);
  const BatchConfig cfg = kConfigs[config];
  cudaError_t e = cfg.unroll == 4 ? launch_phases<4>(t, cfg.blocks_per_sm, s, d)
                                  : launch_phases<2>(t, cfg.blocks_per_sm, s, d);
  if (e != cudaSuccess) return e;
  k_batch_resolve<<<screen_blocks, kThreads, 0, s>>>(t);
  return cudaGetLastError();
}

}  // namespace pcr
