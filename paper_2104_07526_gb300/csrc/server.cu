// Serving loop (include/pcr.h, "Serving"): resident point clouds, frame
// slots and continuous batching of view requests on top of the batched
// renderer (batch.cu).
//
// Device memory comes from one caller-owned arena: frame slots and batch
// workspaces are carved out at creation, clouds are placed first-fit in the
// rest on demand and evicted least-recently-used when room is needed (never
// while a batch in flight reads them).  pcr_server_step is the loop body:
// it retires batches whose completion event has fired, then forms new
// batches from the queued requests, in arrival order, as long as an
// in-flight batch, frame slots and cloud memory are free.  Every batch runs
// on the batched renderer, which sends a view that shares no pass over its
// cloud's points with another through the single-view kernels.  Batches
// rotate over the server's streams (one per in-flight batch unless fewer are
// asked for), so with several streams they overlap on the GPU; requests that
// arrive while others render join the next batch.
// A request's result stays in its frame slot until the caller releases the
// ticket.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <unordered_map>
#include <vector>

#include "../../include/pcr.h"
#include "launch.h"

namespace pcr {
namespace {

constexpr uint64_t kAlign = 256;
constexpr uint32_t kMaxInflight = 8;

uint64_t align_up(uint64_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

double now_us() {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over offsets [0, size) of the arena, with coalescing.
class FreeList {
 public:
  void reset(uint64_t size) {
    free_.clear();
    if (size > 0) free_[0] = size;
  }
  bool alloc(uint64_t bytes, uint64_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const uint64_t rest = it->second - bytes;
      const uint64_t at = it->first + bytes;
      free_.erase(it);
      if (rest > 0) free_[at] = rest;
      return true;
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }

 private:
  std::map<uint64_t, uint64_t> free_;
};

struct Cloud {
  const void* host = nullptr;   // source of uploads (host registrations)
  const void* device = nullptr; // caller's device copy (device registrations, never evicted)
  uint64_t n = 0;
  uint64_t bytes = 0;
  bool resident = false;
  uint64_t offset = 0;          // in the arena, when resident and host-registered
  uint32_t pins = 0;            // batches in flight that read it
  uint64_t last_use = 0;        // LRU clock
  cudaEvent_t ready = nullptr;  // completion of its latest upload
  bool uploaded_once = false;
};

enum : int { kQueued = 0, kRunning = 1, kDone = 2, kExpired = 3, kCancelled = 4 };

struct Request {
  uint32_t cloud = 0;
  float matrix[16];
  int32_t width = 0, height = 0;
  uint32_t flags = 0;
  int state = kQueued;
  int slot = -1;
  double t_submit = 0, t_launch = 0, t_done = 0;
};

struct Inflight {
  cudaStream_t stream = nullptr;  // borrowed from pcr_server::streams
  cudaEvent_t done = nullptr;
  void* staging = nullptr;  // pinned host copy of the job tables
  void* workspace = nullptr;
  bool busy = false;
  std::vector<uint64_t> tickets;
  std::vector<uint32_t> clouds;
};

}  // namespace

Device ctx_device(pcr_ctx* ctx);
bool ctx_capturing(const pcr_ctx* ctx);

}  // namespace pcr

struct pcr_server {
  pcr::Device dev;
  pcr_server_config cfg;
  char* arena = nullptr;
  uint64_t cloud_base = 0;  // clouds live in [cloud_base, arena_bytes)
  uint64_t slot_bytes = 0, slot_pixels = 0;
  std::vector<uint64_t> slot_offset;
  std::vector<int> free_slots;
  pcr::FreeList mem;
  std::unordered_map<uint32_t, pcr::Cloud> clouds;
  std::unordered_map<uint64_t, pcr::Request> requests;
  std::deque<uint64_t> queue;
  std::deque<uint64_t> finished;  // completed tickets not yet reported by pcr_server_poll_completed
  std::vector<pcr::Inflight> inflight;
  std::vector<cudaStream_t> streams;
  uint64_t next_ticket = 1;
  uint64_t clock = 0;
  pcr_server_stats stats{};
};

namespace {

using pcr::kDone;
using pcr::kCancelled;
using pcr::kExpired;
using pcr::kQueued;
using pcr::kRunning;

// A request that left the server's hands: rendered, expired or cancelled.
bool finished(int state) { return state == kDone || state == kExpired || state == kCancelled; }

struct SlotPtrs {
  unsigned long long* keys;
  uint32_t* image;
  uint32_t* depth;
  unsigned long long* rg;
  unsigned long long* ba;
  uint32_t* hq_image;
};

// Slot layout: keys (8 B/px), depth (4), rg (8), ba (8), image (4), hq image (4).
SlotPtrs slot_ptrs(const pcr_server* s, int slot) {
  char* base = s->arena + s->slot_offset[slot];
  const uint64_t px = s->slot_pixels;
  SlotPtrs p;
  p.keys = reinterpret_cast<unsigned long long*>(base);
  p.rg = reinterpret_cast<unsigned long long*>(base + pcr::align_up(8 * px));
  p.ba = reinterpret_cast<unsigned long long*>(base + 2 * pcr::align_up(8 * px));
  p.depth = reinterpret_cast<uint32_t*>(base + 3 * pcr::align_up(8 * px));
  p.image = reinterpret_cast<uint32_t*>(base + 3 * pcr::align_up(8 * px) + pcr::align_up(4 * px));
  p.hq_image = reinterpret_cast<uint32_t*>(base + 3 * pcr::align_up(8 * px) + 2 * pcr::align_up(4 * px));
  return p;
}

const void* cloud_points(const pcr_server* s, const pcr::Cloud& c) {
  return c.device ? c.device : static_cast<const void*>(s->arena + s->cloud_base + c.offset);
}

// Make room for `bytes` by evicting least-recently-used unpinned clouds.
bool reserve(pcr_server* s, uint64_t bytes, uint64_t* off) {
  for (;;) {
    if (s->mem.alloc(bytes, off)) return true;
    pcr::Cloud* victim = nullptr;
    for (auto& kv : s->clouds) {
      pcr::Cloud& c = kv.second;
      if (c.resident && !c.device && c.pins == 0 && (!victim || c.last_use < victim->last_use)) victim = &c;
    }
    if (!victim) return false;
    s->mem.release(victim->offset, pcr::align_up(victim->bytes));
    victim->resident = false;
    ++s->stats.evictions;
  }
}

pcr_status retire(pcr_server* s, uint32_t* completed) {
  for (pcr::Inflight& f : s->inflight) {
    if (!f.busy) continue;
    const cudaError_t q = cudaEventQuery(f.done);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return PCR_ERR_CUDA;
    const double t = pcr::now_us();
    for (uint64_t tk : f.tickets) {
      pcr::Request& r = s->requests[tk];
      r.state = kDone;
      r.t_done = t;
      s->finished.push_back(tk);
      ++s->stats.completed;
      s->stats.points_rendered += s->clouds[r.cloud].n;
      if (completed) ++*completed;
    }
    for (uint32_t c : f.clouds) --s->clouds[c].pins;
    f.tickets.clear();
    f.clouds.clear();
    f.busy = false;
  }
  return PCR_OK;
}

// Requests still queued deadline_us after their submission expire: they
// leave the queue unrendered and are reported like finished ones.  The queue
// is in arrival order, so they are at its front.
void expire(pcr_server* s, uint32_t* completed) {
  if (s->cfg.deadline_us == 0) return;
  const double t = pcr::now_us();
  while (!s->queue.empty()) {
    pcr::Request& r = s->requests[s->queue.front()];
    if (t - r.t_submit < s->cfg.deadline_us) break;
    r.state = kExpired;
    r.t_done = t;
    s->finished.push_back(s->queue.front());
    s->queue.pop_front();
    ++s->stats.expired;
    if (completed) ++*completed;
  }
}

// The clouds a new batch may take requests of, or an empty list for any
// cloud (arrival order with no cloud limit).  Arrival order: filled as the
// queue is walked.  Largest groups: the oldest request's cloud, then the
// clouds with the most queued requests.
std::vector<uint32_t> batch_cloud_choice(const pcr_server* s, uint32_t cloud_cap) {
  std::vector<uint32_t> chosen;
  if (s->cfg.policy != PCR_SERVE_LARGEST_GROUP || s->queue.empty()) return chosen;
  std::unordered_map<uint32_t, uint32_t> count;
  for (uint64_t tk : s->queue) ++count[s->requests.at(tk).cloud];
  const uint32_t oldest = s->requests.at(s->queue.front()).cloud;
  std::vector<std::pair<uint32_t, uint32_t>> by_count(count.begin(), count.end());
  std::sort(by_count.begin(), by_count.end(), [](const auto& a, const auto& b) {
    return a.second != b.second ? a.second > b.second : a.first < b.first;
  });
  chosen.push_back(oldest);
  for (const auto& kv : by_count) {
    if (chosen.size() >= cloud_cap) break;
    if (kv.first != oldest) chosen.push_back(kv.first);
  }
  return chosen;
}

// Form and launch one batch on the free in-flight slot `f`.  Returns
// PCR_OK with nothing launched when no queued request can run now.
pcr_status launch_one(pcr_server* s, pcr::Inflight& f, bool* launched) {
  *launched = false;
  std::vector<uint64_t> take;
  std::vector<uint32_t> batch_clouds;  // distinct cloud ids, in order of first use
  std::vector<uint32_t> uploads;       // clouds this batch uploads
  const uint32_t cloud_cap =
      std::min<uint32_t>(s->cfg.max_batch_clouds ? s->cfg.max_batch_clouds : PCR_BATCH_MAX_CLOUDS,
                         PCR_BATCH_MAX_CLOUDS);
  const std::vector<uint32_t> allowed = batch_cloud_choice(s, cloud_cap);
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    if (take.size() >= s->cfg.max_batch_views || s->free_slots.empty()) break;
    pcr::Request& r = s->requests[*it];
    pcr::Cloud& c = s->clouds[r.cloud];
    const bool in_batch = std::find(batch_clouds.begin(), batch_clouds.end(), r.cloud) != batch_clouds.end();
    const bool excluded = !allowed.empty() && std::find(allowed.begin(), allowed.end(), r.cloud) == allowed.end();
    if (excluded || (!in_batch && batch_clouds.size() >= cloud_cap)) {
      ++it;
      continue;
    }
    if (!c.resident) {
      uint64_t off = 0;
      if (!reserve(s, pcr::align_up(c.bytes), &off)) {  // everything else is pinned: try a later request
        ++it;
        continue;
      }
      c.offset = off;
      c.resident = true;
      uploads.push_back(r.cloud);
    }
    if (!in_batch) {
      batch_clouds.push_back(r.cloud);
      ++c.pins;
    }
    c.last_use = ++s->clock;
    r.slot = s->free_slots.back();
    s->free_slots.pop_back();
    take.push_back(*it);
    it = s->queue.erase(it);
  }
  if (take.empty()) return PCR_OK;

  std::vector<pcr_batch_cloud> bc(batch_clouds.size());
  for (size_t i = 0; i < batch_clouds.size(); ++i) {
    const pcr::Cloud& c = s->clouds[batch_clouds[i]];
    bc[i].points = cloud_points(s, c);
    bc[i].n = c.n;
  }
  std::vector<pcr_batch_view> bv(take.size());
  for (size_t i = 0; i < take.size(); ++i) {
    const pcr::Request& r = s->requests[take[i]];
    pcr_batch_view& v = bv[i];
    std::memcpy(v.matrix, r.matrix, sizeof(v.matrix));
    v.width = r.width;
    v.height = r.height;
    v.cloud = static_cast<uint32_t>(std::find(batch_clouds.begin(), batch_clouds.end(), r.cloud) -
                                    batch_clouds.begin());
    v.flags = r.flags;
    const SlotPtrs p = slot_ptrs(s, r.slot);
    v.keys = (r.flags & PCR_BATCH_BASIC) ? p.keys : nullptr;
    v.image = (r.flags & PCR_BATCH_BASIC) ? p.image : nullptr;
    v.hq_depth = (r.flags & PCR_BATCH_HQ) ? p.depth : nullptr;
    v.hq_rg = (r.flags & PCR_BATCH_HQ) ? p.rg : nullptr;
    v.hq_ba = (r.flags & PCR_BATCH_HQ) ? p.ba : nullptr;
    v.hq_image = (r.flags & PCR_BATCH_HQ) ? p.hq_image : nullptr;
  }
  pcr::batch_build_tables(bc.data(), static_cast<uint32_t>(bc.size()), bv.data(), static_cast<uint32_t>(bv.size()),
                          s->cfg.depth_factor, s->cfg.background_rgba, f.staging,
                          s->cfg.l2_budget_mb ? static_cast<uint64_t>(s->cfg.l2_budget_mb) << 20
                                              : pcr::kServedL2Budget);

  cudaError_t e = cudaSuccess;
  for (uint32_t id : uploads) {
    pcr::Cloud& c = s->clouds[id];
    if (e == cudaSuccess && c.n > 0)
      e = cudaMemcpyAsync(s->arena + s->cloud_base + c.offset, c.host, c.bytes, cudaMemcpyHostToDevice, f.stream);
    if (e == cudaSuccess) e = cudaEventRecord(c.ready, f.stream);
    c.uploaded_once = true;
    ++s->stats.uploads;
    s->stats.bytes_uploaded += c.bytes;
  }
  for (uint32_t id : batch_clouds) {  // an upload issued by another batch stream must finish first
    const pcr::Cloud& c = s->clouds[id];
    if (e == cudaSuccess && !c.device && c.uploaded_once &&
        std::find(uploads.begin(), uploads.end(), id) == uploads.end())
      e = cudaStreamWaitEvent(f.stream, c.ready, 0);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(f.workspace, f.staging, pcr::batch_tables_bytes(), cudaMemcpyHostToDevice, f.stream);
  if (e == cudaSuccess) e = pcr::batch_launch(f.staging, f.workspace, s->cfg.batch_config, f.stream, s->dev);
  if (e == cudaSuccess) e = cudaEventRecord(f.done, f.stream);
  if (e != cudaSuccess) {
    // nothing of this batch is known to have run: its requests go back to the
    // front of the queue, in order, with their slots and cloud pins released
    for (auto it = take.rbegin(); it != take.rend(); ++it) {
      pcr::Request& r = s->requests[*it];
      s->free_slots.push_back(r.slot);
      r.slot = -1;
      s->queue.push_front(*it);
    }
    for (uint32_t id : batch_clouds) --s->clouds[id].pins;
    for (uint32_t id : uploads) {  // their uploads may not have run
      pcr::Cloud& c = s->clouds[id];
      s->mem.release(c.offset, pcr::align_up(c.bytes));
      c.resident = false;
    }
    return PCR_ERR_CUDA;
  }

  const double t = pcr::now_us();
  for (uint64_t tk : take) {
    pcr::Request& r = s->requests[tk];
    r.state = kRunning;
    r.t_launch = t;
  }
  f.tickets = std::move(take);
  f.clouds = std::move(batch_clouds);
  f.busy = true;
  ++s->stats.batches;
  s->stats.views_launched += f.tickets.size();
  *launched = true;
  return PCR_OK;
}

void destroy(pcr_server* s) {
  for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
  for (pcr::Inflight& f : s->inflight) {
    if (f.done) cudaEventDestroy(f.done);
    if (f.staging) cudaFreeHost(f.staging);
  }
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  for (auto& kv : s->clouds)
    if (kv.second.ready) cudaEventDestroy(kv.second.ready);
  delete s;
}

}  // namespace

extern "C" {

pcr_status pcr_server_create(pcr_ctx* ctx, const pcr_server_config* cfg, pcr_server** out) {
  if (!ctx || !cfg || !out || pcr::ctx_capturing(ctx)) return PCR_ERR_ARG;
  *out = nullptr;
  if (!cfg->dev_arena || (reinterpret_cast<uintptr_t>(cfg->dev_arena) & (pcr::kAlign - 1))) return PCR_ERR_ARG;
  if (cfg->max_width < 1 || cfg->max_height < 1 || cfg->max_width > 16384 || cfg->max_height > 16384)
    return PCR_ERR_ARG;
  if (cfg->num_slots < 1 || cfg->max_batch_views < 1 || cfg->max_batch_views > PCR_BATCH_MAX_VIEWS ||
      cfg->max_inflight < 1 || cfg->max_inflight > pcr::kMaxInflight || cfg->streams > cfg->max_inflight ||
      cfg->max_batch_clouds > PCR_BATCH_MAX_CLOUDS)
    return PCR_ERR_ARG;
  if (!(cfg->depth_factor > 0.0f) || !(cfg->depth_factor < 3.0e38f)) return PCR_ERR_ARG;
  if (cfg->batch_config < 0 || cfg->batch_config >= pcr::batch_num_configs()) return PCR_ERR_ARG;
  if (cfg->policy != PCR_SERVE_ARRIVAL && cfg->policy != PCR_SERVE_LARGEST_GROUP) return PCR_ERR_ARG;
  if (cfg->l2_budget_mb > 1024) return PCR_ERR_ARG;
  pcr_server* s = new (std::nothrow) pcr_server();
  if (!s) return PCR_ERR_CUDA;
  s->dev = pcr::ctx_device(ctx);
  s->cfg = *cfg;
  s->arena = static_cast<char*>(cfg->dev_arena);
  s->slot_pixels = static_cast<uint64_t>(cfg->max_width) * cfg->max_height;
  s->slot_bytes = 3 * pcr::align_up(8 * s->slot_pixels) + 3 * pcr::align_up(4 * s->slot_pixels);
  const uint64_t ws_bytes = pcr::align_up(pcr::batch_workspace_bytes());
  const uint64_t fixed = cfg->num_slots * s->slot_bytes + cfg->max_inflight * ws_bytes;
  if (fixed > cfg->arena_bytes) {
    delete s;
    return PCR_ERR_WORKSPACE;
  }
  for (uint32_t i = 0; i < cfg->num_slots; ++i) {
    s->slot_offset.push_back(i * s->slot_bytes);
    s->free_slots.push_back(static_cast<int>(cfg->num_slots - 1 - i));
  }
  s->cloud_base = fixed;
  s->mem.reset(cfg->arena_bytes - fixed);
  const uint64_t ws_base = cfg->num_slots * s->slot_bytes;
  s->inflight.resize(cfg->max_inflight);
  pcr_status st = PCR_OK;
  {
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != s->dev.id) cudaSetDevice(s->dev.id);
    const uint32_t nstreams = cfg->streams ? cfg->streams : cfg->max_inflight;
    for (uint32_t i = 0; i < nstreams && st == PCR_OK; ++i) {
      cudaStream_t sm = nullptr;
      if (cudaStreamCreateWithFlags(&sm, cudaStreamNonBlocking) != cudaSuccess) st = PCR_ERR_CUDA;
      else s->streams.push_back(sm);
    }
    for (uint32_t i = 0; i < cfg->max_inflight && st == PCR_OK; ++i) {
      pcr::Inflight& f = s->inflight[i];
      f.workspace = s->arena + ws_base + i * ws_bytes;
      f.stream = s->streams[i % nstreams];
      if (cudaEventCreateWithFlags(&f.done, cudaEventDisableTiming) != cudaSuccess ||
          cudaHostAlloc(&f.staging, pcr::batch_tables_bytes(), cudaHostAllocDefault) != cudaSuccess)
        st = PCR_ERR_CUDA;
    }
    if (st == PCR_OK && pcr::batch_prewarm(s->dev) != cudaSuccess) st = PCR_ERR_CUDA;
    if (prev >= 0 && prev != s->dev.id) cudaSetDevice(prev);
  }
  if (st != PCR_OK) {
    destroy(s);
    return st;
  }
  *out = s;
  return PCR_OK;
}

pcr_status pcr_server_destroy(pcr_server* s) {
  if (s) destroy(s);
  return PCR_OK;
}

static pcr_status add_cloud(pcr_server* s, uint32_t id, const void* host, const void* device, uint64_t n) {
  if (!s || n > 0xFFFFFFFFull || s->clouds.count(id)) return PCR_ERR_ARG;
  if (n > 0 && !host && !device) return PCR_ERR_ARG;
  if (device && (reinterpret_cast<uintptr_t>(device) & 15)) return PCR_ERR_ARG;
  pcr::Cloud c;
  c.host = host;
  c.device = device;
  c.n = n;
  c.bytes = n * 16;
  c.resident = device != nullptr;
  if (cudaEventCreateWithFlags(&c.ready, cudaEventDisableTiming) != cudaSuccess) return PCR_ERR_CUDA;
  s->clouds[id] = c;
  return PCR_OK;
}

pcr_status pcr_server_add_cloud(pcr_server* s, uint32_t cloud_id, const void* host_points, uint64_t n) {
  return add_cloud(s, cloud_id, host_points, nullptr, n);
}

pcr_status pcr_server_add_device_cloud(pcr_server* s, uint32_t cloud_id, const void* dev_points, uint64_t n) {
  return add_cloud(s, cloud_id, nullptr, dev_points, n);
}

pcr_status pcr_server_submit(pcr_server* s, const pcr_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return PCR_ERR_ARG;
  if (!s->clouds.count(req->cloud_id)) return PCR_ERR_ARG;
  if (req->width < 1 || req->height < 1 || static_cast<uint32_t>(req->width) > s->cfg.max_width ||
      static_cast<uint32_t>(req->height) > s->cfg.max_height)
    return PCR_ERR_ARG;
  if (req->flags == 0 || (req->flags & ~static_cast<uint32_t>(PCR_BATCH_BASIC | PCR_BATCH_HQ))) return PCR_ERR_ARG;
  const pcr::Cloud& c = s->clouds[req->cloud_id];
  if (!c.device && pcr::align_up(c.bytes) > s->cfg.arena_bytes - s->cloud_base) return PCR_ERR_WORKSPACE;  // never fits
  if (s->cfg.max_queue && s->queue.size() >= s->cfg.max_queue) {
    ++s->stats.rejected;
    return PCR_ERR_BUSY;
  }
  pcr::Request r;
  r.cloud = req->cloud_id;
  std::memcpy(r.matrix, req->matrix, sizeof(r.matrix));
  r.width = req->width;
  r.height = req->height;
  r.flags = req->flags;
  r.t_submit = pcr::now_us();
  const uint64_t t = s->next_ticket++;
  s->requests[t] = r;
  s->queue.push_back(t);
  ++s->stats.submitted;
  s->stats.peak_queue = std::max<uint64_t>(s->stats.peak_queue, s->queue.size());
  *ticket = t;
  return PCR_OK;
}

pcr_status pcr_server_step(pcr_server* s, uint32_t* completed) {
  if (!s) return PCR_ERR_ARG;
  if (completed) *completed = 0;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != s->dev.id) cudaSetDevice(s->dev.id);
  pcr_status st = retire(s, completed);
  expire(s, completed);
  for (pcr::Inflight& f : s->inflight) {
    if (st != PCR_OK || s->queue.empty()) break;
    if (f.busy) continue;
    bool launched = false;
    st = launch_one(s, f, &launched);
    if (!launched) break;
  }
  if (prev >= 0 && prev != s->dev.id) cudaSetDevice(prev);
  return st;
}

pcr_status pcr_server_state(pcr_server* s, uint64_t ticket, int* state) {
  if (!s || !state) return PCR_ERR_ARG;
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return PCR_ERR_ARG;
  *state = it->second.state;
  return PCR_OK;
}

pcr_status pcr_server_get_result(pcr_server* s, uint64_t ticket, pcr_server_result* out) {
  if (!s || !out) return PCR_ERR_ARG;
  auto it = s->requests.find(ticket);
  if (it == s->requests.end() || !finished(it->second.state)) return PCR_ERR_ARG;
  const pcr::Request& r = it->second;
  if (r.state != kDone) {  // expired or cancelled: never rendered
    *out = pcr_server_result{};
    out->width = r.width;
    out->height = r.height;
    out->submit_us = r.t_submit;
    out->done_us = r.t_done;
    return PCR_OK;
  }
  const SlotPtrs p = slot_ptrs(s, r.slot);
  out->width = r.width;
  out->height = r.height;
  out->flags = r.flags;
  out->keys = (r.flags & PCR_BATCH_BASIC) ? p.keys : nullptr;
  out->image = (r.flags & PCR_BATCH_BASIC) ? p.image : nullptr;
  out->hq_depth = (r.flags & PCR_BATCH_HQ) ? p.depth : nullptr;
  out->hq_rg = (r.flags & PCR_BATCH_HQ) ? p.rg : nullptr;
  out->hq_ba = (r.flags & PCR_BATCH_HQ) ? p.ba : nullptr;
  out->hq_image = (r.flags & PCR_BATCH_HQ) ? p.hq_image : nullptr;
  out->submit_us = r.t_submit;
  out->launch_us = r.t_launch;
  out->done_us = r.t_done;
  out->points = s->clouds[r.cloud].n;
  return PCR_OK;
}

pcr_status pcr_server_poll_completed(pcr_server* s, uint64_t* tickets, uint32_t capacity, uint32_t* count) {
  if (!s || !count || (capacity > 0 && !tickets)) return PCR_ERR_ARG;
  uint32_t k = 0;
  while (k < capacity && !s->finished.empty()) {
    tickets[k++] = s->finished.front();
    s->finished.pop_front();
  }
  *count = k;
  return PCR_OK;
}

pcr_status pcr_server_cancel(pcr_server* s, uint64_t ticket) {
  if (!s) return PCR_ERR_ARG;
  auto it = s->requests.find(ticket);
  if (it == s->requests.end() || finished(it->second.state)) return PCR_ERR_ARG;
  if (it->second.state == kRunning) return PCR_ERR_BUSY;
  const auto q = std::find(s->queue.begin(), s->queue.end(), ticket);
  if (q == s->queue.end()) return PCR_ERR_ARG;
  s->queue.erase(q);
  it->second.state = kCancelled;
  it->second.t_done = pcr::now_us();
  s->finished.push_back(ticket);
  ++s->stats.cancelled;
  return PCR_OK;
}

pcr_status pcr_server_release(pcr_server* s, uint64_t ticket) {
  if (!s) return PCR_ERR_ARG;
  auto it = s->requests.find(ticket);
  if (it == s->requests.end() || !finished(it->second.state)) return PCR_ERR_ARG;
  if (it->second.state == kDone) s->free_slots.push_back(it->second.slot);
  s->requests.erase(it);
  return PCR_OK;
}

pcr_status pcr_server_stats_get(pcr_server* s, pcr_server_stats* out) {
  if (!s || !out) return PCR_ERR_ARG;
  *out = s->stats;
  out->queued = s->queue.size();
  uint64_t resident = 0, bytes = 0;
  for (const auto& kv : s->clouds)
    if (kv.second.resident && !kv.second.device) {
      ++resident;
      bytes += kv.second.bytes;
    }
  out->resident_clouds = resident;
  out->resident_bytes = bytes;
  return PCR_OK;
}

}  // extern "C"
