// C interface (include/pcr.h): argument checks, context state and launches.
// No exception leaves this file; every entry point returns a pcr_status.
#include <cstdint>
#include <cstring>
#include <new>

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

}  // namespace

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
  *out = c;
  return PCR_OK;
}

pcr_status pcr_destroy(pcr_ctx* ctx) {
  delete ctx;
  return PCR_OK;
}

pcr_status pcr_set_stream(pcr_ctx* ctx, void* cuda_stream) {
  if (!ctx) return PCR_ERR_ARG;
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
  if (!ctx || n > kMaxPoints) return PCR_ERR_ARG;
  if (n > 0 && (!dev_points || !host_points || !aligned(dev_points, 16))) return PCR_ERR_ARG;
  if (n > 0) {
    DeviceScope scope(ctx->dev.id);
    if (!scope.ok()) return PCR_ERR_CUDA;
    const cudaError_t e = cudaMemcpyAsync(dev_points, host_points, n * 16, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return PCR_ERR_CUDA;
  }
  return pcr_upload_points(ctx, dev_points, n);
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
  if (!ctx || variant < PCR_VARIANT_ATOMICMIN || variant > PCR_VARIANT_JUST_SET) return PCR_ERR_ARG;
  if (!view_ready(ctx) || !ctx->keys) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  if (clear) {
    const cudaError_t e = pcr::launch_fill_u64(ctx->keys, pixels(ctx), pcr::kEmptyKey, ctx->stream, ctx->dev);
    if (e != cudaSuccess) return PCR_ERR_CUDA;
  }
  return from_cuda(pcr::launch_render_basic(variant, ctx->points, static_cast<uint32_t>(ctx->n), view_params(ctx),
                                            ctx->keys, ctx->stream, ctx->dev));
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
  if (!ctx) return PCR_ERR_ARG;
  if (bytes == 0) return PCR_OK;
  if (!host_dst || !dev_src) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  cudaError_t e = cudaMemcpyAsync(host_dst, dev_src, bytes, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  return from_cuda(e);
}

pcr_status pcr_synchronize(pcr_ctx* ctx) {
  if (!ctx) return PCR_ERR_ARG;
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
  if (!ctx || n > kMaxPoints || mode < PCR_ORDER_MORTON || mode > PCR_ORDER_SHUFFLE) return PCR_ERR_ARG;
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
  if (!ctx || mode < PCR_ORDER_MORTON || mode > PCR_ORDER_SHUFFLE) return PCR_ERR_ARG;
  if (n > PCR_REORDER_NOALLOC_MAX_POINTS) return PCR_ERR_WORKSPACE;
  if (n == 0) return PCR_OK;
  if (!dev_points || !aligned(dev_points, 16) || (dev_perm_out && !aligned(dev_perm_out, 4))) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  return from_cuda(pcr::launch_reorder_noalloc(static_cast<uint4*>(dev_points), static_cast<uint32_t>(n), seed,
                                               mode, dev_perm_out, ctx->stream, ctx->dev));
}

const char* pcr_status_string(pcr_status status) {
  switch (status) {
    case PCR_OK: return "ok";
    case PCR_ERR_ARG: return "invalid argument";
    case PCR_ERR_CUDA: return "CUDA error";
    case PCR_ERR_WORKSPACE: return "workspace missing or too small";
    case PCR_ERR_TIMEOUT: return "device wait timed out";
    case PCR_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

pcr_status pcr_last_device_error(pcr_ctx* ctx, uint32_t* code) {
  if (!ctx || !code) return PCR_ERR_ARG;
  DeviceScope scope(ctx->dev.id);
  if (!scope.ok()) return PCR_ERR_CUDA;
  return from_cuda(pcr::read_and_clear_error_word(code, ctx->stream));
}

}  // extern "C"
