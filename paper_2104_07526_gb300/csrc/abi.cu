// C interface (include/pcr.h): argument checks, context state and launches.
// No exception leaves this file; every entry point returns a pcr_status.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/pcr.h"
#include "launch.h"

struct pcr_ctx {
  pcr::Device dev;
  cudaStream_t stream = nullptr;
  const uint4* points = nullptr;
  uint64_t n = 0;
  float m[16] = {};
  bool has_matrix = false;
  int width = 0;
  int height = 0;
  unsigned long long* keys = nullptr;
  uint32_t* depth = nullptr;
  unsigned long long* rg = nullptr;
  unsigned long long* ba = nullptr;
  unsigned long long* primary = nullptr;  // HQS1R primary words
  uint32_t* locks = nullptr;              // busy-loop lock words
  uint64_t lock_wait_ns = 100000000ull;
  // Host copy of the tables of every batch workspace this context prepared:
  // a batch launch reads the views it renders through the single-view
  // kernels from it.
  std::unordered_map<const void*, std::vector<unsigned char>> batch_plans;
  // Between pcr_capture_begin and pcr_capture_end: the private stream being
  // recorded (it stands in for `stream`, saved in `captured_stream`).
  cudaStream_t capture = nullptr;
  cudaStream_t captured_stream = nullptr;
};

namespace {

constexpr uint64_t kMaxPoints = 0xFFFFFFFFull;  // indices are 32-bit
constexpr int kMaxViewport = 16384;

// Makes the context's device current for one call and restores the caller's.
class DeviceScope {
 public:
  explicit DeviceScope(int device) : target_(device) {
    if (cudaGetDevice(&prev_) != cudaSuccess) {
      ok_ = false;
      return;
    }
    if (prev_ != target_) ok_ = cudaSetDevice(target_) == cudaSuccess;
  }
  ~DeviceScope() {
    if (ok_ && prev_ >= 0 && prev_ != target_) cudaSetDevice(prev_);
  }
  bool ok() const { return ok_; }

 private:
  int target_;
  int prev_ = -1;
  bool ok_ = true;
};

pcr_status from_cuda(cudaError_t e) { return e == cudaSuccess ? PCR_OK : PCR_ERR_CUDA; }

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

pcr::ViewParams view_params(const pcr_ctx* c) {
  pcr::ViewParams v{};
  for (int k = 0; k < 4; ++k) {
    v.r0[k] = c->m[k];
    v.r1[k] = c->m[4 + k];
    v.r3[k] = c->m[12 + k];
  }
  v.fw = static_cast<float>(c->width);
  v.fh = static_cast<float>(c->height);
  v.width = static_cast<uint32_t>(c->width);
  v.height = static_cast<uint32_t>(c->height);
  return v;
}

uint64_t pixels(const pcr_ctx* c) { return static_cast<uint64_t>(c->width) * static_cast<uint64_t>(c->height); }

bool view_ready(const pcr_ctx* c) { return c->has_matrix && c->width > 0 && c->height > 0; }

// Arguments of pcr_batch_prepare and pcr_batch_tune.
pcr_status check_batch(const pcr_ctx* ctx, const pcr_batch_cloud* clouds, uint32_t num_clouds,
                       const pcr_batch_view* views, uint32_t num_views, float depth_factor, const void* dev_workspace,
                       uint64_t workspace_bytes) {
  if (!ctx || ctx->capture || !clouds || !views) return PCR_ERR_ARG;  // both synchronise: not while capturing
  if (num_clouds == 0 || num_clouds > PCR_BATCH_MAX_CLOUDS || num_views == 0 || num_views > PCR_BATCH_MAX_VIEWS)
    return PCR_ERR_ARG;
  if (!(depth_factor > 0.0f) || !(depth_factor < 3.0e38f)) return PCR_ERR_ARG;
  for (uint32_t c = 0; c < num_clouds; ++c) {
    if (clouds[c].n > kMaxPoints) return PCR_ERR_ARG;
    if (clouds[c].n > 0 && (!clouds[c].points || !aligned(clouds[c].points, 16))) return PCR_ERR_ARG;
  }
  for (uint32_t i = 0; i < num_views; ++i) {
    const pcr_batch_view& v = views[i];
    if (v.cloud >= num_clouds || v.width < 1 || v.height < 1 || v.width > kMaxViewport || v.height > kMaxViewport)
      return PCR_ERR_ARG;
    if (v.flags == 0 || (v.flags & ~static_cast<uint32_t>(PCR_BATCH_BASIC | PCR_BATCH_HQ))) return PCR_ERR_ARG;
    if ((v.flags & PCR_BATCH_BASIC) &&
        (!v.keys || !aligned(v.keys, 8) || (v.image && !aligned(v.image, 4))))
      return PCR_ERR_ARG;
    if ((v.flags & PCR_BATCH_HQ) && (!v.hq_depth || !aligned(v.hq_depth, 4) || !v.hq_rg || !aligned(v.hq_rg, 8) ||
                                     !v.hq_ba || !aligned(v.hq_ba, 8) || (v.hq_image && !aligned(v.hq_image, 4))))
      return PCR_ERR_ARG;
  }
  if (!dev_workspace || !aligned(dev_workspace, 256) || workspace_bytes < pcr::batch_workspace_bytes())
    return PCR_ERR_WORKSPACE;
  return PCR_OK;
}

// L2 budgets (MB of framebuffer one pass over a cloud may touch) the batch
// tuner tries; the middle one is pcr_batch_prepare's.
constexpr int kTuneBudgetsMb[] = {64, 96, 128};
constexpr int kNumTuneBudgets = 3;

// "<device name> sm<count>": the GPU a tuning result belongs to.
std::string gpu_id(const pcr::Device& d) {
  cudaDeviceProp prop{};
  std::string name = cudaGetDeviceProperties(&prop, d.id) == cudaSuccess ? prop.name : "unknown";
  for (char& ch : name)
    if (ch == '"' || ch == '\\' || ch < 32) ch = '_';
  return name + " sm" + std::to_string(d.num_sms);
}

// The shape of a batch: cloud sizes and each view's size, flags and cloud
// (not its camera), as counts and a 64-bit FNV-1a hash.
std::string batch_shape_key(const pcr_batch_cloud* clouds, uint32_t num_clouds, const pcr_batch_view* views,
                            uint32_t num_views) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&h](uint64_t v) {
    for (int k = 0; k < 8; ++k) {
      h ^= (v >> (8 * k)) & 0xFF;
      h *= 1099511628211ull;
    }
  };
  for (uint32_t c = 0; c < num_clouds; ++c) mix(clouds[c].n);
  for (uint32_t i = 0; i < num_views; ++i) {
    mix(static_cast<uint64_t>(views[i].width) << 32 | static_cast<uint32_t>(views[i].height));
    mix(static_cast<uint64_t>(views[i].flags) << 32 | views[i].cloud);
  }
  char buf[64];
  std::snprintf(buf, sizeof(buf), "c%uv%u-%016llx", num_clouds, num_views, static_cast<unsigned long long>(h));
  return buf;
}

// The integer after `"name": ` in a line of the cache, if present.
bool json_int(const std::string& line, const char* name, long long* v) {
  const std::string tag = std::string("\"") + name + "\": ";
  const size_t at = line.find(tag);
  if (at == std::string::npos) return false;
  char* end = nullptr;
  *v = std::strtoll(line.c_str() + at + tag.size(), &end, 10);
  return end != line.c_str() + at + tag.size();
}

// The cache is a file of JSON lines, one per tuned (GPU, shape); the last
// line for a pair wins.
bool read_tuning(const char* path, const std::string& gpu, const std::string& shape, int* budget_mb, int* config) {
  std::FILE* f = std::fopen(path, "r");
  if (!f) return false;
  bool found = false;
  char buf[1024];
  const std::string want_gpu = "\"gpu\": \"" + gpu + "\"", want_shape = "\"shape\": \"" + shape + "\"";
  while (std::fgets(buf, sizeof(buf), f)) {
    const std::string line(buf);
    long long b = 0, c = 0;
    if (line.find(want_gpu) == std::string::npos || line.find(want_shape) == std::string::npos) continue;
    if (!json_int(line, "budget_mb", &b) || !json_int(line, "config", &c)) continue;
    bool known = false;
    for (int k = 0; k < kNumTuneBudgets; ++k) known = known || b == kTuneBudgetsMb[k];
    if (!known || c < 0 || c >= pcr::batch_num_configs()) continue;
    *budget_mb = static_cast<int>(b);
    *config = static_cast<int>(c);
    found = true;
  }
  std::fclose(f);
  return found;
}

void fill_tuning(pcr_batch_tuning* out, int budget_mb, int config, int from_cache, int tried, double best_ms,
                 double default_ms) {
  out->l2_budget_mb = static_cast<uint32_t>(budget_mb);
  out->config = config;
  out->threads = static_cast<uint32_t>(pcr::batch_config_threads(config));
  out->unroll1 = static_cast<uint32_t>(pcr::batch_config_unroll(config, 0));
  out->unroll2 = static_cast<uint32_t>(pcr::batch_config_unroll(config, 1));
  out->single_colors = pcr::batch_config_single_colors(config) ? 1u : 0u;
  out->from_cache = static_cast<uint32_t>(from_cache);
  out->tried = static_cast<uint32_t>(tried);
  out->best_ms = best_ms;
  out->default_ms = default_ms;
}

void write_tuning(const char* path, const std::string& gpu, const std::string& shape, const pcr_batch_tuning& t) {
  std::FILE* f = std::fopen(path, "a");
  if (!f) return;  // the cache is an optimisation: a read-only location only loses it
  std::fprintf(f,
               "{\"gpu\": \"%s\", \"shape\": \"%s\", \"budget_mb\": %u, \"config\": %d, \"threads\": %u, "
               "\"unroll1\": %u, \"unroll2\": %u, \"ms\": %.4f, \"default_ms\": %.4f}\n",
               gpu.c_str(), shape.c_str(), t.l2_budget_mb, t.config, t.threads, t.unroll1, t.unroll2, t.best_ms,
               t.default_ms);
  std::fclose(f);
}

// The host tables of a workspace this context prepared (nullptr if none),
// and room for them (nullptr if out of memory).
const void* find_plan(const pcr_ctx* ctx, const void* ws) {
  const auto it = ctx->batch_plans.find(ws);
  return it == ctx->batch_plans.end() ? nullptr : it->second.data();
}

void* plan_for(pcr_ctx* ctx, const void* ws) {
  try {
    std::vector<unsigned char>& v = ctx->batch_plans[ws];
    v.resize(pcr::batch_tables_bytes());
    return v.data();
  } catch (const std::bad_alloc&) {
    ctx->batch_plans.erase(ws);
    return nullptr;
  }
}

// Time one launch configuration on the prepared workspace: one warm-up
// launch, then three timed ones; *ms per launch.
cudaError_t time_batch(const void* ws, int config, pcr_ctx* ctx, cudaEvent_t a, cudaEvent_t b, double* ms) {
  const void* plan = find_plan(ctx, ws);
  if (!plan) return cudaErrorInvalidValue;
  cudaError_t e = pcr::batch_launch(plan, ws, config, ctx->stream, ctx->dev);
  if (e == cudaSuccess) e = cudaEventRecord(a, ctx->stream);
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) e = pcr::batch_launch(plan, ws, config, ctx->stream, ctx->dev);
  if (e == cudaSuccess) e = cudaEventRecord(b, ctx->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  *ms = t / 3.0;
  return e;
}

}  // namespace

namespace pcr {
Device ctx_device(pcr_ctx* ctx) { return ctx->dev; }
bool ctx_capturing(const pcr_ctx* ctx) { return ctx->capture != nullptr; }
}  // namespace pcr

extern "C" {

pcr_status pcr_create(pcr_ctx** out, int device) {
  if (!out) return PCR_ERR_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess) {
    cudaGetLastError();
    return PCR_ERR_CUDA;
  }
  if (device < 0 || device >= count) return PCR_ERR_ARG;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0)
    return PCR_ERR_CUDA;
  pcr_ctx* c = new (std::nothrow) pcr_ctx();
  if (!c) return PCR_ERR_CUDA;
  c->dev.id = device;
  c->dev.num_sms = sms;
  pcr::forget_noalloc_scratch(device);
  *out = c;
  return PCR_OK;
}

pcr_status pcr_destroy(pcr_ctx* ctx) {
  if (ctx && ctx->capture) {  // an unfinished capture is dropped
    cudaGraph_t graph = nullptr;
    cudaStreamEndCapture(ctx->capture, &graph);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(ctx->capture);
    cudaGetLastError();
  }
  delete ctx;
  return PCR_OK;
}

pcr_status pcr_capture_begin(pcr_ctx* ctx) {
  if (!ctx || ctx->capture) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  // occupancy queries (and the module loads they may cause) happen before
  // recording starts
  pcr::prewarm_single_view(ctx->dev);
  if (pcr::batch_prewarm(ctx->dev) != cudaSuccess) return PCR_ERR_CUDA;
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return PCR_ERR_CUDA;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaStreamDestroy(cs);
    return PCR_ERR_CUDA;
  }
  ctx->captured_stream = ctx->stream;
  ctx->stream = ctx->capture = cs;
  return PCR_OK;
}

pcr_status pcr_capture_end(pcr_ctx* ctx, void** graph_exec) {
  if (!ctx || !graph_exec || !ctx->capture) return PCR_ERR_ARG;
  *graph_exec = nullptr;
  DeviceScope scope(ctx->dev.id);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->capture, &graph);
  cudaStreamDestroy(ctx->capture);
  ctx->stream = ctx->captured_stream;
  ctx->capture = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess || !scope.ok()) {
    cudaGetLastError();
    return PCR_ERR_CUDA;
  }
  *graph_exec = exec;
  return PCR_OK;
}

pcr_status pcr_set_stream(pcr_ctx* ctx, void* cuda_stream) {
  if (!ctx || ctx->capture) return PCR_ERR_ARG;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return PCR_OK;
}

pcr_status pcr_upload_points(pcr_ctx* ctx, const void* dev_points, uint64_t n) {
  if (!ctx || n > kMaxPoints) return PCR_ERR_ARG;
  if (n > 0 && (!dev_points || !aligned(dev_points, 16))) return PCR_ERR_ARG;
  ctx->points = static_cast<const uint4*>(dev_points);
  ctx->n = n;
  return PCR_OK;
}

pcr_status pcr_upload_points_from_host(pcr_ctx* ctx, void* dev_points, const void* host_points, uint64_t n) {
  if (!ctx || ctx->capture || n > kMaxPoints) return PCR_ERR_ARG;
  if (n > 0 && (!dev_points || !host_points || !aligned(dev_points, 16))) return PCR_ERR_ARG;
  if (n > 0) {
    DeviceScope scope(ctx->dev.id);
    if (!scope.ok()) return PCR_ERR_CUDA;
    const cudaError_t e = cudaMemcpyAsync(dev_points, host_points, n * 16, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return PCR_ERR_CUDA;
  }
  return pcr_upload_points(ctx, dev_points, n);
}

namespace {
// Device address of a byte of pinned, mapped host memory, or nullptr.
void* mapped_address(const void* host) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost) return nullptr;
  void* dev = nullptr;
  if (cudaHostGetDevicePointer(&dev, const_cast<void*>(host), 0) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return dev;
}
}  // namespace

pcr_status pcr_upload_points_mapped(pcr_ctx* ctx, const void* host_points, uint64_t n) {
  if (!ctx || n > kMaxPoints) return PCR_ERR_ARG;
  if (n == 0) return pcr_upload_points(ctx, nullptr, 0);
  if (!host_points || !aligned(host_points, 16)) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  // Both ends must be pinned and mapped, and map to one contiguous range.
  const uint64_t last = n * 16 - 1;
  char* first_dev = static_cast<char*>(mapped_address(host_points));
  char* last_dev = static_cast<char*>(mapped_address(static_cast<const char*>(host_points) + last));
  if (!first_dev || !last_dev || last_dev != first_dev + last) return PCR_ERR_ARG;
  return pcr_upload_points(ctx, first_dev, n);
}

pcr_status pcr_set_matrix(pcr_ctx* ctx, const float m[16]) {
  if (!ctx || !m) return PCR_ERR_ARG;
  std::memcpy(ctx->m, m, sizeof(ctx->m));
  ctx->has_matrix = true;
  return PCR_OK;
}

pcr_status pcr_set_viewport(pcr_ctx* ctx, int width, int height) {
  if (!ctx || width < 1 || height < 1 || width > kMaxViewport || height > kMaxViewport) return PCR_ERR_ARG;
  ctx->width = width;
  ctx->height = height;
  return PCR_OK;
}

pcr_status pcr_set_framebuffer(pcr_ctx* ctx, void* dev_keys, void* dev_hq_depth, void* dev_hq_rg, void* dev_hq_ba) {
  if (!ctx) return PCR_ERR_ARG;
  if ((dev_keys && !aligned(dev_keys, 8)) || (dev_hq_depth && !aligned(dev_hq_depth, 4)) ||
      (dev_hq_rg && !aligned(dev_hq_rg, 8)) || (dev_hq_ba && !aligned(dev_hq_ba, 8)))
    return PCR_ERR_ARG;
  ctx->keys = static_cast<unsigned long long*>(dev_keys);
  ctx->depth = static_cast<uint32_t*>(dev_hq_depth);
  ctx->rg = static_cast<unsigned long long*>(dev_hq_rg);
  ctx->ba = static_cast<unsigned long long*>(dev_hq_ba);
  return PCR_OK;
}

pcr_status pcr_clear(pcr_ctx* ctx, int what) {
  if (!ctx || what <= 0 || (what & ~(PCR_CLEAR_KEYS | PCR_CLEAR_HQ)) || ctx->width <= 0) return PCR_ERR_ARG;
  if ((what & PCR_CLEAR_KEYS) && !ctx->keys) return PCR_ERR_ARG;
  if ((what & PCR_CLEAR_HQ) && (!ctx->depth || !ctx->rg || !ctx->ba)) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  cudaError_t e = cudaSuccess;
  if (what & PCR_CLEAR_KEYS) e = pcr::launch_fill_u64(ctx->keys, pixels(ctx), pcr::kEmptyKey, ctx->stream, ctx->dev);
  if (e == cudaSuccess && (what & PCR_CLEAR_HQ))
    e = pcr::launch_clear_hq(ctx->depth, ctx->rg, ctx->ba, pixels(ctx), ctx->stream, ctx->dev);
  return from_cuda(e);
}

pcr_status pcr_render_basic(pcr_ctx* ctx, int variant, int clear) {
  if (!ctx || variant < PCR_VARIANT_ATOMICMIN || variant > PCR_VARIANT_BUSY_LOOP) return PCR_ERR_ARG;
  if (!view_ready(ctx) || !ctx->keys) return PCR_ERR_ARG;
  const bool busy = variant == PCR_VARIANT_BUSY_LOOP;
  if (busy && !ctx->locks) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  cudaError_t e = cudaSuccess;
  if (clear) e = pcr::launch_fill_u64(ctx->keys, pixels(ctx), pcr::kEmptyKey, ctx->stream, ctx->dev);
  if (e == cudaSuccess && clear && busy) e = pcr::launch_fill_u32(ctx->locks, pixels(ctx), 0u, ctx->stream, ctx->dev);
  if (e != cudaSuccess) return PCR_ERR_CUDA;
  const uint32_t n = static_cast<uint32_t>(ctx->n);
  if (busy)
    return from_cuda(pcr::launch_render_busy(ctx->points, n, view_params(ctx), ctx->keys, ctx->locks,
                                             ctx->lock_wait_ns, ctx->stream, ctx->dev));
  return from_cuda(pcr::launch_render_basic(variant, ctx->points, n, view_params(ctx), ctx->keys, ctx->stream,
                                            ctx->dev));
}

pcr_status pcr_render_rgb(pcr_ctx* ctx, int variant, int clear) {
  if (!ctx || variant < PCR_VARIANT_ATOMICMIN || variant > PCR_VARIANT_JUST_SET) return PCR_ERR_ARG;
  if (!view_ready(ctx) || !ctx->keys) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  if (clear) {
    const cudaError_t e = pcr::launch_fill_u64(ctx->keys, pixels(ctx), pcr::kEmptyKey, ctx->stream, ctx->dev);
    if (e != cudaSuccess) return PCR_ERR_CUDA;
  }
  return from_cuda(pcr::launch_render_rgb(variant, ctx->points, static_cast<uint32_t>(ctx->n), view_params(ctx),
                                          ctx->keys, ctx->stream, ctx->dev));
}

pcr_status pcr_set_lock_buffer(pcr_ctx* ctx, void* dev_locks, uint32_t wait_limit_us) {
  if (!ctx || (dev_locks && !aligned(dev_locks, 4))) return PCR_ERR_ARG;
  ctx->locks = static_cast<uint32_t*>(dev_locks);
  ctx->lock_wait_ns = 1000ull * (wait_limit_us ? wait_limit_us : 100000u);
  return PCR_OK;
}

pcr_status pcr_render_hq(pcr_ctx* ctx, float depth_factor, int variant, int clear) {
  if (!ctx || variant < PCR_VARIANT_ATOMICMIN || variant > PCR_VARIANT_DEDUP_EARLYZ) return PCR_ERR_ARG;
  if (!(depth_factor > 0.0f) || !(depth_factor < 3.0e38f)) return PCR_ERR_ARG;
  if (!view_ready(ctx) || !ctx->depth || !ctx->rg || !ctx->ba) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  const uint32_t n = static_cast<uint32_t>(ctx->n);
  const pcr::ViewParams v = view_params(ctx);
  cudaError_t e = cudaSuccess;
  if (clear) e = pcr::launch_clear_hq(ctx->depth, ctx->rg, ctx->ba, pixels(ctx), ctx->stream, ctx->dev);
  if (e == cudaSuccess) e = pcr::launch_hq_depth(variant, ctx->points, n, v, ctx->depth, ctx->stream, ctx->dev);
  if (e == cudaSuccess)
    e = pcr::launch_hq_color(variant, ctx->points, n, v, depth_factor, ctx->depth, ctx->rg, ctx->ba, ctx->stream,
                             ctx->dev);
  return from_cuda(e);
}

pcr_status pcr_set_hq1r_buffer(pcr_ctx* ctx, void* dev_primary) {
  if (!ctx || (dev_primary && !aligned(dev_primary, 8))) return PCR_ERR_ARG;
  ctx->primary = static_cast<unsigned long long*>(dev_primary);
  return PCR_OK;
}

pcr_status pcr_render_hq1r(pcr_ctx* ctx, float depth_factor, int variant, int clear) {
  if (!ctx || variant < PCR_VARIANT_ATOMICMIN || variant > PCR_VARIANT_DEDUP_EARLYZ) return PCR_ERR_ARG;
  if (!(depth_factor > 0.0f) || !(depth_factor < 3.0e38f)) return PCR_ERR_ARG;
  if (!view_ready(ctx) || !ctx->depth || !ctx->rg || !ctx->ba || !ctx->primary) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  const uint32_t n = static_cast<uint32_t>(ctx->n);
  const pcr::ViewParams v = view_params(ctx);
  cudaError_t e = cudaSuccess;
  if (clear) {
    e = pcr::launch_clear_hq(ctx->depth, ctx->rg, ctx->ba, pixels(ctx), ctx->stream, ctx->dev);
    if (e == cudaSuccess) e = pcr::launch_fill_u64(ctx->primary, pixels(ctx), 0ull, ctx->stream, ctx->dev);
  }
  if (e == cudaSuccess) e = pcr::launch_hq_depth(variant, ctx->points, n, v, ctx->depth, ctx->stream, ctx->dev);
  if (e == cudaSuccess)
    e = pcr::launch_hq1r_color(variant, ctx->points, n, v, depth_factor, ctx->depth, ctx->primary, ctx->rg, ctx->ba,
                               ctx->stream, ctx->dev);
  return from_cuda(e);
}

pcr_status pcr_resolve(pcr_ctx* ctx, int mode, void* dev_rgba_out, uint32_t background_rgba) {
  if (!ctx || !dev_rgba_out || !aligned(dev_rgba_out, 4) || !view_ready(ctx)) return PCR_ERR_ARG;
  uint32_t* out = static_cast<uint32_t*>(dev_rgba_out);
  if (mode == PCR_RESOLVE_BASIC) {
    if (!ctx->keys) return PCR_ERR_ARG;
    DeviceScope scope(ctx->dev.id);
    if (!scope.ok()) return PCR_ERR_CUDA;
    return from_cuda(pcr::launch_resolve_basic(ctx->keys, pixels(ctx), ctx->points, static_cast<uint32_t>(ctx->n),
                                               background_rgba, out, ctx->stream, ctx->dev));
  }
  if (mode == PCR_RESOLVE_HQ1R) {
    if (!ctx->rg || !ctx->ba || !ctx->primary) return PCR_ERR_ARG;
    DeviceScope scope(ctx->dev.id);
    if (!scope.ok()) return PCR_ERR_CUDA;
    return from_cuda(pcr::launch_resolve_hq1r(ctx->primary, ctx->rg, ctx->ba, pixels(ctx), background_rgba, out,
                                              ctx->stream, ctx->dev));
  }
  if (mode == PCR_RESOLVE_RGB) {
    if (!ctx->keys) return PCR_ERR_ARG;
    DeviceScope scope(ctx->dev.id);
    if (!scope.ok()) return PCR_ERR_CUDA;
    return from_cuda(pcr::launch_resolve_rgb(ctx->keys, pixels(ctx), background_rgba, out, ctx->stream, ctx->dev));
  }
  if (mode == PCR_RESOLVE_HQ) {
    if (!ctx->rg || !ctx->ba) return PCR_ERR_ARG;
    DeviceScope scope(ctx->dev.id);
    if (!scope.ok()) return PCR_ERR_CUDA;
    return from_cuda(
        pcr::launch_resolve_hq(ctx->rg, ctx->ba, pixels(ctx), background_rgba, out, ctx->stream, ctx->dev));
  }
  return PCR_ERR_ARG;
}

pcr_status pcr_download(pcr_ctx* ctx, void* host_dst, const void* dev_src, uint64_t bytes) {
  if (!ctx || ctx->capture) return PCR_ERR_ARG;
  if (bytes == 0) return PCR_OK;
  if (!host_dst || !dev_src) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  cudaError_t e = cudaMemcpyAsync(host_dst, dev_src, bytes, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  return from_cuda(e);
}

pcr_status pcr_synchronize(pcr_ctx* ctx) {
  if (!ctx || ctx->capture) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  return from_cuda(cudaStreamSynchronize(ctx->stream));
}

pcr_status pcr_reorder_workspace_size(uint64_t n, uint64_t* bytes) {
  if (!bytes || n > kMaxPoints) return PCR_ERR_ARG;
  *bytes = pcr::reorder_workspace_bytes(n);
  return PCR_OK;
}

pcr_status pcr_reorder_morton_shuffle128(pcr_ctx* ctx, void* dev_points, uint64_t n, uint64_t seed, int mode,
                                         void* dev_workspace, uint64_t workspace_bytes, uint32_t* dev_perm_out) {
  if (!ctx || ctx->capture || n > kMaxPoints || mode < PCR_ORDER_MORTON || mode > PCR_ORDER_MORTON63_SHUFFLE128)
    return PCR_ERR_ARG;
  if (n == 0) return PCR_OK;
  if (!dev_points || !aligned(dev_points, 16) || (dev_perm_out && !aligned(dev_perm_out, 4))) return PCR_ERR_ARG;
  if (!dev_workspace || !aligned(dev_workspace, 256) || workspace_bytes < pcr::reorder_workspace_bytes(n))
    return PCR_ERR_WORKSPACE;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  return from_cuda(pcr::launch_reorder(static_cast<uint4*>(dev_points), static_cast<uint32_t>(n), seed, mode,
                                       dev_workspace, dev_perm_out, ctx->stream, ctx->dev));
}

pcr_status pcr_reorder_morton_shuffle128_noalloc(pcr_ctx* ctx, void* dev_points, uint64_t n, uint64_t seed,
                                                 int mode, uint32_t* dev_perm_out) {
  if (!ctx || ctx->capture || mode < PCR_ORDER_MORTON || mode > PCR_ORDER_MORTON63_SHUFFLE128) return PCR_ERR_ARG;
  if (n > PCR_REORDER_NOALLOC_MAX_POINTS) return PCR_ERR_WORKSPACE;
  if (n == 0) return PCR_OK;
  if (!dev_points || !aligned(dev_points, 16) || (dev_perm_out && !aligned(dev_perm_out, 4))) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  return from_cuda(pcr::launch_reorder_noalloc(static_cast<uint4*>(dev_points), static_cast<uint32_t>(n), seed,
                                               mode, dev_perm_out, ctx->stream, ctx->dev));
}

pcr_status pcr_batch_workspace_size(uint64_t* bytes) {
  if (!bytes) return PCR_ERR_ARG;
  *bytes = pcr::batch_workspace_bytes();
  return PCR_OK;
}

pcr_status pcr_batch_num_configs(int* count) {
  if (!count) return PCR_ERR_ARG;
  *count = pcr::batch_num_configs();
  return PCR_OK;
}

pcr_status pcr_batch_prepare(pcr_ctx* ctx, const pcr_batch_cloud* clouds, uint32_t num_clouds,
                             const pcr_batch_view* views, uint32_t num_views, float depth_factor,
                             uint32_t background_rgba, void* dev_workspace, uint64_t workspace_bytes) {
  const pcr_status st = check_batch(ctx, clouds, num_clouds, views, num_views, depth_factor, dev_workspace,
                                    workspace_bytes);
  if (st != PCR_OK) return st;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  void* plan = plan_for(ctx, dev_workspace);
  if (!plan) return PCR_ERR_CUDA;  // no host memory for the tables
  return from_cuda(pcr::batch_prepare(clouds, num_clouds, views, num_views, depth_factor, background_rgba, plan,
                                      dev_workspace, ctx->stream));
}

pcr_status pcr_batch_tune(pcr_ctx* ctx, const pcr_batch_cloud* clouds, uint32_t num_clouds,
                          const pcr_batch_view* views, uint32_t num_views, float depth_factor,
                          uint32_t background_rgba, void* dev_workspace, uint64_t workspace_bytes,
                          const char* cache_path, pcr_batch_tuning* out) {
  if (!out) return PCR_ERR_ARG;
  const pcr_status st = check_batch(ctx, clouds, num_clouds, views, num_views, depth_factor, dev_workspace,
                                    workspace_bytes);
  if (st != PCR_OK) return st;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  *out = pcr_batch_tuning{};
  void* plan = plan_for(ctx, dev_workspace);
  if (!plan) return PCR_ERR_CUDA;  // no host memory for the tables
  const std::string gpu = gpu_id(ctx->dev);
  const std::string shape = batch_shape_key(clouds, num_clouds, views, num_views);
  int cached_budget = 0, cached_config = -1;
  if (cache_path && read_tuning(cache_path, gpu, shape, &cached_budget, &cached_config)) {
    const cudaError_t e = pcr::batch_prepare(clouds, num_clouds, views, num_views, depth_factor, background_rgba,
                                             plan, dev_workspace, ctx->stream,
                                             static_cast<uint64_t>(cached_budget) << 20);
    if (e != cudaSuccess) return PCR_ERR_CUDA;
    fill_tuning(out, cached_budget, cached_config, 1, 0, 0.0, 0.0);
    return PCR_OK;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return PCR_ERR_CUDA;
  }
  cudaError_t e = pcr::batch_prewarm(ctx->dev);
  int best_budget = kTuneBudgetsMb[1], best_config = 0, tried = 0;
  double best_ms = 0.0, default_ms = 0.0;
  for (int bi = 0; bi < kNumTuneBudgets && e == cudaSuccess; ++bi) {
    const int budget = kTuneBudgetsMb[bi];
    e = pcr::batch_prepare(clouds, num_clouds, views, num_views, depth_factor, background_rgba, plan,
                           dev_workspace, ctx->stream, static_cast<uint64_t>(budget) << 20);
    for (int c = 0; c < pcr::batch_num_configs() && e == cudaSuccess; ++c) {
      double ms = 0.0;
      e = time_batch(dev_workspace, c, ctx, a, b, &ms);
      if (e != cudaSuccess) break;
      ++tried;
      if (budget == kTuneBudgetsMb[1] && c == 0) default_ms = ms;
      if (tried == 1 || ms < best_ms) {
        best_ms = ms;
        best_budget = budget;
        best_config = c;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e == cudaSuccess)  // leave the workspace prepared with the winner
    e = pcr::batch_prepare(clouds, num_clouds, views, num_views, depth_factor, background_rgba, plan,
                           dev_workspace, ctx->stream, static_cast<uint64_t>(best_budget) << 20);
  if (e != cudaSuccess) return PCR_ERR_CUDA;
  fill_tuning(out, best_budget, best_config, 0, tried, best_ms, default_ms);
  if (cache_path) write_tuning(cache_path, gpu, shape, *out);
  return PCR_OK;
}

pcr_status pcr_batch_launch(pcr_ctx* ctx, const void* dev_workspace, int config) {
  if (!ctx || !dev_workspace || !aligned(dev_workspace, 256) || config < 0 || config >= pcr::batch_num_configs())
    return PCR_ERR_ARG;
  const void* plan = find_plan(ctx, dev_workspace);
  if (!plan) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  return from_cuda(pcr::batch_launch(plan, dev_workspace, config, ctx->stream, ctx->dev));
}

pcr_status pcr_batch_launch_count(pcr_ctx* ctx, const void* dev_workspace, int config, int* count) {
  if (!ctx || !dev_workspace || !count || config < 0 || config >= pcr::batch_num_configs()) return PCR_ERR_ARG;
  const void* plan = find_plan(ctx, dev_workspace);
  if (!plan) return PCR_ERR_ARG;
  *count = pcr::batch_launch_count(plan, config);
  return PCR_OK;
}

pcr_status pcr_batch_autotune(pcr_ctx* ctx, const void* dev_workspace, int* config) {
  if (!ctx || ctx->capture || !dev_workspace || !config || !aligned(dev_workspace, 256)) return PCR_ERR_ARG;
  const void* plan = find_plan(ctx, dev_workspace);
  if (!plan) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return PCR_ERR_CUDA;
  }
  int best = 0;
  float best_ms = 0.0f;
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < pcr::batch_num_configs() && e == cudaSuccess; ++c) {
    e = pcr::batch_launch(plan, dev_workspace, c, ctx->stream, ctx->dev);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(a, ctx->stream);
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep)
      e = pcr::batch_launch(plan, dev_workspace, c, ctx->stream, ctx->dev);
    if (e == cudaSuccess) e = cudaEventRecord(b, ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && (c == 0 || ms < best_ms)) {
      best = c;
      best_ms = ms;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return PCR_ERR_CUDA;
  *config = best;
  return PCR_OK;
}

pcr_status pcr_batch_capture(pcr_ctx* ctx, const void* dev_workspace, int config, void** graph_exec) {
  if (!ctx || ctx->capture || !dev_workspace || !graph_exec || !aligned(dev_workspace, 256) || config < 0 ||
      config >= pcr::batch_num_configs())
    return PCR_ERR_ARG;
  *graph_exec = nullptr;
  const void* plan = find_plan(ctx, dev_workspace);
  if (!plan) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  cudaError_t e = pcr::batch_prewarm(ctx->dev);  // occupancy queries happen before the capture
  if (e != cudaSuccess) return PCR_ERR_CUDA;
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return PCR_ERR_CUDA;
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const cudaError_t le = pcr::batch_launch(plan, dev_workspace, config, cs, ctx->dev);
    e = cudaStreamEndCapture(cs, &graph);
    if (le != cudaSuccess) e = le;
  }
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return PCR_ERR_CUDA;
  *graph_exec = exec;
  return PCR_OK;
}

pcr_status pcr_graph_launch(pcr_ctx* ctx, void* graph_exec) {
  if (!ctx || !graph_exec) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  return from_cuda(cudaGraphLaunch(static_cast<cudaGraphExec_t>(graph_exec), ctx->stream));
}

pcr_status pcr_graph_destroy(void* graph_exec) {
  if (graph_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(graph_exec));
  return PCR_OK;
}

pcr_status pcr_check_division(pcr_ctx* ctx, uint32_t w_first, uint32_t w_count, const uint32_t* dev_c_bits,
                              uint32_t c_first, uint32_t c_count, uint32_t c_step, float size, uint64_t out[5]) {
  if (!ctx || ctx->capture || !out || (c_count > 0 && !dev_c_bits && c_step == 0) ||
      !(size > 0.0f && size <= 16384.0f))
    return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  return from_cuda(pcr::check_division(w_first, w_count, dev_c_bits, c_first, c_count, c_step, size, out,
                                       ctx->stream, ctx->dev));
}

const char* pcr_status_string(pcr_status status) {
  switch (status) {
    case PCR_OK: return "ok";
    case PCR_ERR_ARG: return "invalid argument";
    case PCR_ERR_CUDA: return "CUDA error";
    case PCR_ERR_WORKSPACE: return "workspace missing or too small";
    case PCR_ERR_TIMEOUT: return "device wait timed out";
    case PCR_ERR_UNSUPPORTED: return "unsupported";
    case PCR_ERR_BUSY: return "queue full";
    default: return "unknown status";
  }
}

pcr_status pcr_debug_counters(pcr_ctx* ctx, uint64_t out[4]) {
  if (!ctx || ctx->capture || !out) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  bool available = false;
  const cudaError_t e = pcr::read_and_clear_debug_counts(out, ctx->stream, &available);
  if (!available) return PCR_ERR_UNSUPPORTED;
  return from_cuda(e);
}

pcr_status pcr_last_device_error(pcr_ctx* ctx, uint32_t* code) {
  if (!ctx || ctx->capture || !code) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  uint32_t batch = 0, reorder = 0;
  cudaError_t e = pcr::read_and_clear_error_word(code, ctx->stream);
  if (e == cudaSuccess) e = pcr::read_and_clear_batch_error_word(&batch, ctx->stream);
  if (e == cudaSuccess) e = pcr::read_and_clear_reorder_error_word(&reorder, ctx->stream);
  *code |= batch | reorder;
  return from_cuda(e);
}

}  // extern "C"
