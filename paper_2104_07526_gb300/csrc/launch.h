// Host-side launchers shared between the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pcr.h"
#include "common.cuh"

namespace pcr {

// Launch geometry: persistent grids sized from the SM count.
struct Device {
  int id = 0;
  int num_sms = 0;
};

cudaError_t launch_fill_u64(unsigned long long* p, uint64_t count, unsigned long long value, cudaStream_t s,
                            const Device& d);
cudaError_t launch_clear_hq(uint32_t* depth, unsigned long long* rg, unsigned long long* ba, uint64_t npx,
                            cudaStream_t s, const Device& d);
cudaError_t launch_render_rgb(int variant, const uint4* pts, uint32_t n, const ViewParams& v,
                              unsigned long long* keys, cudaStream_t s, const Device& d);
cudaError_t launch_render_busy(const uint4* pts, uint32_t n, const ViewParams& v, unsigned long long* keys,
                               uint32_t* locks, uint64_t limit_ns, cudaStream_t s, const Device& d);
cudaError_t launch_fill_u32(uint32_t* p, uint64_t count, uint32_t value, cudaStream_t s, const Device& d);
cudaError_t launch_resolve_rgb(const unsigned long long* keys, uint64_t npx, uint32_t background, uint32_t* out,
                               cudaStream_t s, const Device& d);
cudaError_t launch_render_basic(int variant, const uint4* pts, uint32_t n, const ViewParams& v,
                                unsigned long long* keys, cudaStream_t s, const Device& d);
cudaError_t launch_hq_depth(int variant, const uint4* pts, uint32_t n, const ViewParams& v, uint32_t* depth,
                            cudaStream_t s, const Device& d);
cudaError_t launch_hq_color(int variant, const uint4* pts, uint32_t n, const ViewParams& v, float depth_factor,
                            const uint32_t* depth, unsigned long long* rg, unsigned long long* ba, cudaStream_t s,
                            const Device& d);
cudaError_t launch_resolve_basic(const unsigned long long* keys, uint64_t npx, const uint4* pts, uint32_t n,
                                 uint32_t background, uint32_t* out, cudaStream_t s, const Device& d);
cudaError_t launch_hq1r_color(int variant, const uint4* pts, uint32_t n, const ViewParams& v, float depth_factor,
                              const uint32_t* depth, unsigned long long* primary, unsigned long long* rg,
                              unsigned long long* ba, cudaStream_t s, const Device& d);
cudaError_t launch_resolve_hq1r(const unsigned long long* primary, const unsigned long long* rg,
                                const unsigned long long* ba, uint64_t npx, uint32_t background, uint32_t* out,
                                cudaStream_t s, const Device& d);
cudaError_t launch_resolve_hq(const unsigned long long* rg, const unsigned long long* ba, uint64_t npx,
                              uint32_t background, uint32_t* out, cudaStream_t s, const Device& d);
cudaError_t read_and_clear_error_word(uint32_t* out, cudaStream_t s);
// Debug builds: the error words of the batch and reorder kernels (0, with no
// device access, in release builds).
cudaError_t read_and_clear_batch_error_word(uint32_t* out, cudaStream_t s);
cudaError_t read_and_clear_reorder_error_word(uint32_t* out, cudaStream_t s);
// Run the occupancy queries of the single-view kernels the batch launches
// (before a capture).
void prewarm_single_view(const Device& d);
// Debug builds: the geometry kernels' counters (render.cu); *available is
// false in release builds.
cudaError_t read_and_clear_debug_counts(uint64_t out[4], cudaStream_t s, bool* available);
// Division check behind pcr_check_division (selfcheck.cu); synchronous.
cudaError_t check_division(uint32_t w_first, uint32_t w_count, const uint32_t* c_bits, uint32_t c_first,
                           uint32_t c_count, uint32_t c_step, float size, uint64_t out[5], cudaStream_t s,
                           const Device& d);

// Batched rendering (batch.cu).  Tables live in the caller's workspace;
// views are grouped by cloud.
constexpr uint32_t kBatchMaxClouds = PCR_BATCH_MAX_CLOUDS;
constexpr uint32_t kBatchMaxViews = PCR_BATCH_MAX_VIEWS;

struct BatchHeader {
  uint32_t num_clouds;
  uint32_t num_views;
  uint64_t total_pixels;  // sum of view sizes
  uint32_t hq_views;
  uint32_t background;
  float depth_factor;
  uint32_t num_groups[2];  // per geometry phase
  uint32_t pad;
  uint64_t total_slots[2];  // per phase: sum over groups of the group's cloud size, padded to 128 points
};

// A group is a set of views of one cloud rendered in one pass over the
// cloud's points; its framebuffers fit the L2 budget.  order[] lists the
// group's view indices.
struct BatchGroup {
  uint32_t cloud;
  uint32_t first;  // into the phase's order[]
  uint32_t count;
  uint32_t pad;
  uint64_t first_slot;  // offset of this group's pass in the phase's padded sequence
};

struct BatchCloud {
  const uint4* pts;
  uint32_t n;
  uint32_t pad;
};

struct BatchView {
  ViewParams vp;
  uint32_t cloud;
  uint32_t flags;
  unsigned long long* keys;
  uint32_t* image;
  uint32_t* depth;
  unsigned long long* rg;
  unsigned long long* ba;
  uint32_t* hq_image;
  uint64_t first_pixel;  // offset of this view in the concatenated pixels
};

uint64_t batch_workspace_bytes();
// Size of the job tables, and building them into caller-provided host
// memory (e.g. pinned staging for an asynchronous copy into a workspace).
uint64_t batch_tables_bytes();
// l2_budget: framebuffer bytes one pass over a cloud may touch (the views of
// a cloud are packed into passes that fit it).
void batch_build_tables(const pcr_batch_cloud* clouds, uint32_t num_clouds, const pcr_batch_view* views,
                        uint32_t num_views, float depth_factor, uint32_t background, void* host_tables,
                        uint64_t l2_budget);
// A batch alone on the GPU (pcr_batch_prepare) packs passes into 96 MB of the
// 129 MB L2; the server, whose batches may run two at a time, into 64 MB.
constexpr uint64_t kBatchL2Budget = 96ull << 20;
constexpr uint64_t kServedL2Budget = 64ull << 20;
int batch_num_configs();
// Build the tables into host_tables (batch_tables_bytes()), copy them into
// the workspace and wait for the copy.
cudaError_t batch_prepare(const pcr_batch_cloud* clouds, uint32_t num_clouds, const pcr_batch_view* views,
                          uint32_t num_views, float depth_factor, uint32_t background, void* host_tables,
                          void* workspace, cudaStream_t s, uint64_t l2_budget = kBatchL2Budget);
// Threads per block and points per lane (phase 0 or 1) of a launch
// configuration, and whether it adds every HQ view's colours single-view.
int batch_config_threads(int config);
int batch_config_unroll(int config, int phase);
bool batch_config_single_colors(int config);
// host_tables: the host copy of the tables in `workspace` (the single-view
// launches read their views from it during the call).
cudaError_t batch_launch(const void* host_tables, const void* workspace, int config, cudaStream_t s,
                         const Device& d);
// Kernel launches batch_launch makes for these tables and configuration.
int batch_launch_count(const void* host_tables, int config);
// Run the occupancy queries of every configuration once (before a capture).
cudaError_t batch_prewarm(const Device& d);

// Vertex order (reorder.cu).
uint64_t reorder_workspace_bytes(uint64_t n);
cudaError_t launch_reorder(uint4* pts, uint32_t n, uint64_t seed, int mode, void* workspace, uint32_t* perm_out,
                           cudaStream_t s, const Device& d);
// The same reorder on the library's fixed scratch array (no allocation);
// the caller has made d's device current and checked n against the limit.
cudaError_t launch_reorder_noalloc(uint4* pts, uint32_t n, uint64_t seed, int mode, uint32_t* perm_out,
                                   cudaStream_t s, const Device& d);
// Drop the cached scratch address of a device (a new context may follow a
// device reset).
void forget_noalloc_scratch(int device);

}  // namespace pcr
