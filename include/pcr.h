/*
 * pcr.h: C interface of a CUDA library (sm_103a) for compute-based point
 * cloud rendering, after Schuetz, Kerbl and Wimmer, "Rendering Point Clouds
 * with Compute Shaders and Vertex Order Optimization" (EGSR 2021).
 *
 * What it computes:
 *  - Sec. 3.1: every point is transformed by a 4x4 matrix, mapped to a pixel
 *    and written with a 64-bit atomic minimum of (depth bits << 32 | point
 *    index) into a key buffer with one word per pixel; a resolve pass turns
 *    keys into colours.
 *  - Sec. 3.2 to 3.4: the same result with an early depth test, a warp-wide
 *    reduction, or full warp deduplication in front of the atomic.
 *  - Sec. 3.5: the high-quality variant: a depth pass, then a colour pass
 *    that sums the colours of all points within a depth band of the nearest
 *    one, then a resolve that averages.
 *  - Sec. 3.5.1: the single-atomic high-quality form (HQS1R); Sec. 3.1 with
 *    the colour-payload key as its listing prints it; Sec. 2 and 5: the
 *    just-set and busy-loop comparison kernels.
 *  - Sec. 4 and 5: Morton order (30-bit, or the paper's 63-bit), shuffled
 *    Morton order (batches of 128 points) and a random shuffle, as a
 *    one-time reordering of the point buffer.
 *  - Many clouds and views rendered together (pcr_batch_*), and a serving
 *    loop over resident clouds with continuous batching (pcr_server_*).
 *
 * Conventions, for every entry point:
 *  - Every call returns a pcr_status.  No C++ exception crosses this
 *    interface and no call aborts the process.
 *  - The caller owns all device memory.  The library borrows pointers for
 *    the duration of the work it launches and never frees them.  It
 *    allocates no device buffers; the context is host memory, and the graphs
 *    and events some calls create hold only driver resources.
 *  - Calls that launch GPU work are asynchronous on the context's stream
 *    (see pcr_set_stream).  Arguments are checked before anything is
 *    launched; a call that returns PCR_ERR_ARG or PCR_ERR_WORKSPACE has
 *    launched nothing.
 *  - A context is used from one host thread at a time.
 *
 * Point record: 16 bytes, 16-byte aligned: float x, y, z, then uint32 rgba
 * with r in the low byte (Sec. 5 gives the same size: 796M points in
 * 12.7 GB).  Indices are 32-bit, so a cloud holds at most 2^32 - 1 points.
 */
#ifndef PCR_H
#define PCR_H

#include <stdint.h>

#if defined(__GNUC__)
#define PCR_API __attribute__((visibility("default")))
#else
#define PCR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int pcr_status;

enum {
    PCR_OK = 0,
    PCR_ERR_ARG = -1,          /* bad argument; nothing was launched */
    PCR_ERR_CUDA = -2,         /* a CUDA call failed (no device, launch error, ...) */
    PCR_ERR_WORKSPACE = -3,    /* workspace missing or too small; nothing was launched */
    PCR_ERR_TIMEOUT = -4,      /* reserved: bounded device-side waits report through
                                  pcr_last_device_error (PCR_DEVICE_ERROR_WAIT_TIMEOUT),
                                  since launches return before the kernel runs */
    PCR_ERR_UNSUPPORTED = -5,  /* valid request this build does not provide */
    PCR_ERR_BUSY = -6          /* a server's queue is full (pcr_server_config.max_queue);
                                  nothing was queued */
};

/* Render variants (Sec. 3.1 to 3.4, and the method list of Sec. 5).  Every
 * variant except PCR_VARIANT_JUST_SET leaves a bit-identical key buffer. */
enum {
    PCR_VARIANT_ATOMICMIN = 0,     /* Sec. 3.1: one 64-bit atomicMin per visible point */
    PCR_VARIANT_EARLYZ = 1,        /* Sec. 3.2: read the pixel first, atomic only if smaller */
    PCR_VARIANT_DEDUP = 2,         /* Sec. 3.4: one atomic per distinct pixel per warp */
    PCR_VARIANT_DEDUP_EARLYZ = 3,  /* Sec. 3.4 with the early test ("dedup" in Sec. 5) */
    PCR_VARIANT_REDUCE = 4,        /* Sec. 3.3: all-equal warp reduction, else pairwise */
    PCR_VARIANT_REDUCE_EARLYZ = 5, /* Sec. 3.3 with the early test */
    PCR_VARIANT_JUST_SET = 6,      /* Sec. 5 "just-set": non-atomic store, no depth test;
                                      a speed floor, not a correct renderer */
    PCR_VARIANT_BUSY_LOOP = 7      /* Sec. 2 and Sec. 5 "busy-loop" (Guenther et al.): early test,
                                      then lock the pixel (compare-and-swap), update, unlock;
                                      pcr_render_basic only, needs pcr_set_lock_buffer */
};

enum {
    PCR_RESOLVE_BASIC = 0,  /* Sec. 3.1: key buffer -> colour of the winning point */
    PCR_RESOLVE_HQ = 1,     /* Sec. 3.5: colour sums -> truncating average */
    PCR_RESOLVE_HQ1R = 2,   /* Sec. 3.5.1: packed primary + fallback sums -> truncating average */
    PCR_RESOLVE_RGB = 3     /* Sec. 3.1: colour-payload keys (pcr_render_rgb) -> their colour */
};

enum {
    PCR_CLEAR_KEYS = 1,     /* key buffer to all ones (empty) */
    PCR_CLEAR_HQ = 2        /* HQ depth to +inf bits, HQ sums to 0 */
};

enum {
    PCR_ORDER_MORTON = 0,            /* Sec. 5 "Morton" */
    PCR_ORDER_MORTON_SHUFFLE128 = 1, /* Sec. 4 and Sec. 5 "Shuffled Morton" */
    PCR_ORDER_SHUFFLE = 2,           /* Sec. 5 "Shuffled" */
    PCR_ORDER_MORTON63 = 3,          /* Sec. 5 "Morton" with the paper's 21 levels (63-bit code) */
    PCR_ORDER_MORTON63_SHUFFLE128 = 4 /* Sec. 4 "Shuffled Morton" over the 63-bit Morton order */
};

/* Bits of the device-side error word (pcr_last_device_error). */
enum {
    PCR_DEVICE_ERROR_KEY_RANGE = 1,    /* a resolve found a key naming a point outside the cloud */
    PCR_DEVICE_ERROR_WAIT_TIMEOUT = 2, /* a busy-loop lock wait gave up (a point was dropped) */
    PCR_DEVICE_ERROR_BOUNDS = 4        /* debug builds: a geometry kernel (single-view or batch) computed a
                                          pixel outside its viewport (the point was dropped), or a reorder
                                          kernel met an index or destination outside the cloud (the access
                                          was skipped); release builds never set it */
};

typedef struct pcr_ctx pcr_ctx;

/* Create a context bound to CUDA device `device`.  Host allocation only.
 * Errors: PCR_ERR_ARG if out is NULL; PCR_ERR_CUDA if the device does not
 * exist or cannot be queried. */
PCR_API pcr_status pcr_create(pcr_ctx **out, int device);

/* Destroy a context (NULL is accepted).  Does not synchronise its stream. */
PCR_API pcr_status pcr_destroy(pcr_ctx *ctx);

/* Use `cuda_stream` (a cudaStream_t, e.g. PyTorch's current stream) for all
 * later work of this context.  NULL selects the legacy default stream.  The
 * library never synchronises a stream except in pcr_synchronize,
 * pcr_download and pcr_last_device_error. */
PCR_API pcr_status pcr_set_stream(pcr_ctx *ctx, void *cuda_stream);

/* Borrow a device point buffer of n records (16-byte aligned, n < 2^32) for
 * the following render and resolve calls.  No copy is made.  n = 0 is
 * allowed (renders then write nothing).  Errors: PCR_ERR_ARG on a NULL or
 * misaligned pointer with n > 0, or n >= 2^32. */
PCR_API pcr_status pcr_upload_points(pcr_ctx *ctx, const void *dev_points, uint64_t n);

/* Copy n records from host memory into the caller's device buffer
 * `dev_points` (asynchronous on the stream; pinned host memory makes it
 * truly asynchronous), then borrow it as pcr_upload_points does.  Same
 * errors as pcr_upload_points, plus PCR_ERR_CUDA if the copy fails. */
PCR_API pcr_status pcr_upload_points_from_host(pcr_ctx *ctx, void *dev_points, const void *host_points, uint64_t n);

/* Borrow n records that stay in pinned host memory (allocated by
 * cudaHostAlloc / cudaMallocHost, or registered by cudaHostRegister, and
 * mapped into the device's address space): the following renders read them
 * over the host link, each render once, with no device copy.  On a Grace
 * host the link (NVLink-C2C) is about as fast as a cudaMemcpyAsync of the
 * same bytes, so a basic frame rendered this way costs the transfer alone,
 * while copy-then-render costs the transfer plus the render.  HQ frames read
 * the points twice; copy those first.  The buffer must stay pinned and
 * unchanged until the work that reads it has finished.  Errors: PCR_ERR_ARG
 * on a NULL or misaligned pointer with n > 0, on n >= 2^32, or when the first
 * or the last record is not in pinned, mapped host memory (plain pageable
 * memory and device memory are refused); PCR_ERR_CUDA if the device cannot be
 * selected. */
PCR_API pcr_status pcr_upload_points_mapped(pcr_ctx *ctx, const void *host_points, uint64_t n);

/* Sec. 3.1 "worldViewProj": a row-major 4x4 float matrix with
 * clip = M (x, y, z, 1)^T.  Only rows 0, 1 and 3 are used: clip.w is the
 * linear depth and there is no near or far plane test.  The matrix is copied.
 * Errors: PCR_ERR_ARG if m is NULL. */
PCR_API pcr_status pcr_set_matrix(pcr_ctx *ctx, const float m[16]);

/* Framebuffer size in pixels, 1..16384 each.  Pixel p = x + y * width with
 * row 0 at the bottom.  Errors: PCR_ERR_ARG out of range. */
PCR_API pcr_status pcr_set_viewport(pcr_ctx *ctx, int width, int height);

/* Borrow the caller's framebuffer storage, each sized for the viewport:
 *   dev_keys      uint64[width*height]  (Sec. 3.1 key buffer), 8-byte aligned
 *   dev_hq_depth  uint32[width*height]  (Sec. 3.5 depth buffer), 4-byte aligned
 *   dev_hq_rg     uint64[width*height]  (Sec. 3.5 r << 32 | g sums)
 *   dev_hq_ba     uint64[width*height]  (Sec. 3.5 b << 32 | count sums)
 * Any may be NULL if the matching render mode is not used; a render that
 * needs a NULL buffer returns PCR_ERR_ARG.  The buffers must not overlap. */
PCR_API pcr_status pcr_set_framebuffer(pcr_ctx *ctx, void *dev_keys, void *dev_hq_depth, void *dev_hq_rg,
                               void *dev_hq_ba);

/* Start a frame (Sec. 3, Fig. "pipeline": buffers are reset before the
 * geometry passes).  `what` is a bit set of PCR_CLEAR_KEYS and PCR_CLEAR_HQ.
 * Errors: PCR_ERR_ARG for an empty or unknown bit set, a missing viewport or
 * a missing buffer. */
PCR_API pcr_status pcr_clear(pcr_ctx *ctx, int what);

/* Sec. 3.1 to 3.4: render the borrowed points into the key buffer.  With
 * clear != 0 the key buffer is first set to all ones (empty); with clear == 0
 * the points are merged into what the buffer holds (a minimum, so several
 * calls over parts of a cloud give the same buffer as one call over all of
 * it, provided index payloads do not collide).  Key of point i:
 * float_bits(w) << 32 | i.  PCR_VARIANT_BUSY_LOOP also needs the lock words
 * of pcr_set_lock_buffer (clear != 0 zeroes them too) and leaves the same
 * buffer as the atomic variants unless a lock wait ran out (see
 * pcr_set_lock_buffer).  Errors: PCR_ERR_ARG for an unknown variant, a
 * missing matrix, viewport, key buffer or (BUSY_LOOP) lock buffer. */
PCR_API pcr_status pcr_render_basic(pcr_ctx *ctx, int variant, int clear);

/* Sec. 3.5: depth pass (32-bit minimum of float_bits(w)), then colour pass:
 * each visible point with w <= float(depth[p]) * depth_factor (float32
 * product; the paper uses 1.01) adds (r << 32 | g) to rg[p] and
 * (b << 32 | 1) to ba[p] with 64-bit integer adds.  clear != 0 first sets
 * depth to +inf and the sums to 0.  `variant` selects the form of the depth
 * pass (ATOMICMIN, EARLYZ, DEDUP, DEDUP_EARLYZ); with every variant but
 * ATOMICMIN the colour pass also sums the colours of same-pixel points
 * within a warp before the adds.  Results do not depend on the variant.  Channel sums are exact while each stays below
 * 2^32 (about 16.8M points per pixel at full intensity).  Errors: PCR_ERR_ARG
 * for a bad variant or depth_factor (not finite or <= 0), missing matrix,
 * viewport or HQ buffers. */
PCR_API pcr_status pcr_render_hq(pcr_ctx *ctx, float depth_factor, int variant, int clear);

/* Sec. 3.1 with the key exactly as Listing "basic" prints it: each visible
 * point offers (float_bits(w) << 24) | (rgba & 0xFFFFFF) to the key buffer,
 * whose minimum keeps the nearest point and, at equal depth, the smallest
 * 24-bit colour.  The key buffer of pcr_set_framebuffer is used; resolve with
 * PCR_RESOLVE_RGB.  Variants as pcr_render_basic except BUSY_LOOP; every
 * variant but JUST_SET leaves the same buffer.  clear != 0 first sets the
 * keys to all ones.  Errors: PCR_ERR_ARG for a bad variant or a missing
 * matrix, viewport or key buffer. */
PCR_API pcr_status pcr_render_rgb(pcr_ctx *ctx, int variant, int clear);

/* Attach the per-pixel lock words of PCR_VARIANT_BUSY_LOOP: uint32[width *
 * height] device memory, caller-owned, 4-byte aligned, all zero between
 * renders (pcr_render_basic with clear != 0 zeroes them; every lock a render
 * takes it gives back).  NULL detaches.  wait_limit_us bounds each lock wait
 * (0 = 100000 us): a wait that runs out sets PCR_DEVICE_ERROR_WAIT_TIMEOUT,
 * drops that point and makes the other waits of the launch give up at once,
 * so the launch always ends.  Errors: PCR_ERR_ARG if misaligned. */
PCR_API pcr_status pcr_set_lock_buffer(pcr_ctx *ctx, void *dev_locks, uint32_t wait_limit_us);

/* Borrow the primary buffer of the single-atomic high-quality variant
 * (Sec. 3.5.1, "HQS1R"): uint64[width*height], 8-byte aligned, holding
 * r << 50 | g << 36 | b << 22 | count (14, 14, 14 and 22 bits; see
 * pcr_render_hq1r).  Its fallback sums live in the dev_hq_rg / dev_hq_ba
 * buffers of pcr_set_framebuffer (same 32-bit layout as HQS).  NULL detaches
 * it.  Errors: PCR_ERR_ARG if misaligned. */
PCR_API pcr_status pcr_set_hq1r_buffer(pcr_ctx *ctx, void *dev_primary);

/* Sec. 3.5.1, "HQS1R": the depth pass of pcr_render_hq, then a colour pass
 * with one 64-bit atomic add per contributing point (or per group of
 * same-pixel points of a warp, with every variant but ATOMICMIN) into the primary
 * word.  The paper's 16-16-16-16 pattern leaves 2^16 - 256 counts of margin
 * for adds that land on a full word before it is reset; a GB300 can have
 * more adds than that in flight on one pixel, so, as the paper allows, the
 * pattern here is 14-14-14-22: a word holds at most 64 points and the count
 * has about 4.2M of margin.  The add whose result would hold more than 64
 * points moves the previous contents and its own colours into the fallback
 * sums and resets the word; adds that land while a word is past 64 points go
 * to the fallback.  Every contribution is counted exactly once, so the
 * combined sums, and the PCR_RESOLVE_HQ1R image, equal those of
 * pcr_render_hq.  clear != 0 first sets depth to +inf, the primary words and
 * the fallback sums to 0.  Errors: as pcr_render_hq, plus PCR_ERR_ARG without
 * a primary buffer. */
PCR_API pcr_status pcr_render_hq1r(pcr_ctx *ctx, float depth_factor, int variant, int clear);

/* Screen pass, writing uint32 rgba per pixel into dev_rgba_out
 * (4-byte aligned, width*height words).
 *   PCR_RESOLVE_BASIC (Sec. 3.1): the rgba word of the point whose index the
 *     key holds; background_rgba where the key is all ones or names no point
 *     of the borrowed cloud.
 *   PCR_RESOLVE_HQ (Sec. 3.5): r = (rg >> 32) / count, g = (rg & 0xffffffff)
 *     / count, b = (ba >> 32) / count with truncating division, each clamped
 *     to 255, alpha 255; background_rgba where count is 0.
 *   PCR_RESOLVE_HQ1R (Sec. 3.5.1): the same average over the primary word's
 *     fields plus the fallback sums.
 * Errors: PCR_ERR_ARG for an unknown mode, NULL output or missing buffers. */
PCR_API pcr_status pcr_resolve(pcr_ctx *ctx, int mode, void *dev_rgba_out, uint32_t background_rgba);

/* Copy `bytes` from device memory to host memory on the context's stream and
 * wait for it.  Errors: PCR_ERR_ARG on NULL pointers with bytes > 0,
 * PCR_ERR_CUDA if the copy fails. */
PCR_API pcr_status pcr_download(pcr_ctx *ctx, void *host_dst, const void *dev_src, uint64_t bytes);

/* Wait for all work queued on the context's stream.  Reports PCR_ERR_CUDA
 * if any of it failed. */
PCR_API pcr_status pcr_synchronize(pcr_ctx *ctx);

/* Bytes of device workspace pcr_reorder_morton_shuffle128 needs for n
 * points (host-only computation, no CUDA call).  Errors: PCR_ERR_ARG if bytes
 * is NULL or n >= 2^32. */
PCR_API pcr_status pcr_reorder_workspace_size(uint64_t n, uint64_t *bytes);

/* Sec. 4 and Sec. 5: reorder a device point buffer in place.
 *   PCR_ORDER_MORTON: stable sort by a 30-bit Morton code (10 bits per axis;
 *     x in bit 3i+2, y in 3i+1, z in 3i) over the cube whose corner is the
 *     minimum of the bounds and whose side is their largest extent; a
 *     coordinate quantises to floor((v - min) * (1024 / extent)) clamped to
 *     [0, 1023]; a zero or non-finite extent gives every point code 0.
 *   PCR_ORDER_MORTON_SHUFFLE128: the Morton order cut into batches of 128
 *     points (the last may be shorter); batch b gets key = high 32 bits of
 *     output b of SplitMix64 seeded with `seed`; batches are stably sorted by
 *     key and keep their inner order.
 *   PCR_ORDER_SHUFFLE: point i gets key = high 32 bits of SplitMix64 output
 *     i; points are stably sorted by key.
 *   PCR_ORDER_MORTON63: as PCR_ORDER_MORTON with the paper's 21 levels: a
 *     63-bit code, 21 bits per axis, floor((v - min) * (2^21 / extent))
 *     clamped to [0, 2^21 - 1].  Its top 30 bits are the 30-bit code.
 *   PCR_ORDER_MORTON63_SHUFFLE128: the batches of PCR_ORDER_MORTON_SHUFFLE128
 *     over the PCR_ORDER_MORTON63 order.
 * dev_points: n records, 16-byte aligned.  dev_workspace: at least the
 * pcr_reorder_workspace_size bytes, 256-byte aligned; its contents are
 * scratch.  dev_perm_out: NULL or uint32[n] (overlapping neither the points
 * nor the workspace; the call may also use it as scratch before it writes
 * the result), receives perm[new] = old.
 * Errors: PCR_ERR_ARG for a bad mode, pointer or n; PCR_ERR_WORKSPACE if
 * workspace_bytes is too small or the workspace is NULL. */
PCR_API pcr_status pcr_reorder_morton_shuffle128(pcr_ctx *ctx, void *dev_points, uint64_t n, uint64_t seed, int mode,
                                         void *dev_workspace, uint64_t workspace_bytes, uint32_t *dev_perm_out);

/* ------------------------------------------------------------------------ */
/* Batched rendering: many (cloud, view, resolution) jobs at once.  The paper  */
/* renders one view per dispatch (Sec. 5 notes the per-dispatch overhead and   */
/* the cost of many small buffers, Sec. 5.4); this interface renders all views */
/* of several clouds in one sequence of four kernels that can be captured as   */
/* one CUDA graph, reading each cloud's points once per phase for all of its   */
/* views.                                                                      */
/* ------------------------------------------------------------------------ */

#define PCR_BATCH_MAX_CLOUDS 256u
#define PCR_BATCH_MAX_VIEWS 256u

enum {
    PCR_BATCH_BASIC = 1,  /* basic frame: key buffer (dedup + early-z) and image */
    PCR_BATCH_HQ = 2      /* high-quality frame: depth, sums and image */
};

typedef struct pcr_batch_cloud {
    const void *points;   /* device, n 16-byte records, 16-byte aligned */
    uint64_t n;           /* < 2^32 */
} pcr_batch_cloud;

typedef struct pcr_batch_view {
    float matrix[16];     /* row-major, as pcr_set_matrix */
    int32_t width;        /* 1..16384 */
    int32_t height;       /* 1..16384 */
    uint32_t cloud;       /* index into the clouds array */
    uint32_t flags;       /* PCR_BATCH_BASIC and/or PCR_BATCH_HQ */
    void *keys;           /* BASIC: uint64[w*h], 8-byte aligned */
    void *image;          /* BASIC: uint32[w*h] rgba, or NULL to skip the resolve */
    void *hq_depth;       /* HQ: uint32[w*h] */
    void *hq_rg;          /* HQ: uint64[w*h] */
    void *hq_ba;          /* HQ: uint64[w*h] */
    void *hq_image;       /* HQ: uint32[w*h] rgba, or NULL to skip the resolve */
} pcr_batch_view;

/* Bytes of device workspace a batch needs (host-only computation). */
PCR_API pcr_status pcr_batch_workspace_size(uint64_t *bytes);

/* Number of launch configurations pcr_batch_launch accepts (0 .. n-1);
 * pcr_batch_autotune and pcr_batch_tune pick among them.  Configuration c
 * runs the geometry phases with 256 << ((c >> 2) & 1) threads per block and
 * (c & 2 ? 2 : 4), (c & 1 ? 2 : 4) points per lane; with c & 8 every HQ
 * view's colours are added by the single-view colour pass instead of
 * phase 2.  0 is the default. */
PCR_API pcr_status pcr_batch_num_configs(int *count);

/* Describe a batch: copy the job tables (clouds, views grouped by cloud)
 * into dev_workspace (256-byte aligned, at least pcr_batch_workspace_size
 * bytes) on the context's stream, and wait for the copy.  The arrays are
 * read during the call only; the buffers they point to are borrowed by every
 * later launch of this workspace.  Each view gets the frames its flags name,
 * with the results of pcr_render_basic(clear) + pcr_resolve(BASIC) and of
 * pcr_render_hq(depth_factor, clear) + pcr_resolve(HQ), bit for bit (the
 * same for every exact variant; the passes use the early depth test).  The
 * views of each cloud are packed into passes over its points whose
 * framebuffers fit 96 MB of the L2 cache (a larger view gets a pass of its
 * own).  A view alone in its pass shares no point loads and is rendered by
 * the single-view kernels (in the keys-and-depth phase only when it asks
 * for one of the two frames).  The context keeps a host copy of the tables
 * (about 52 KB per workspace, until pcr_destroy), which pcr_batch_launch
 * reads for those views.  Errors: PCR_ERR_ARG for counts of 0 or above the maxima, a bad cloud
 * index, size, flags, pointer or alignment, or a bad depth_factor;
 * PCR_ERR_WORKSPACE for a missing or small workspace. */
PCR_API pcr_status pcr_batch_prepare(pcr_ctx *ctx, const pcr_batch_cloud *clouds, uint32_t num_clouds,
                                     const pcr_batch_view *views, uint32_t num_views, float depth_factor,
                                     uint32_t background_rgba, void *dev_workspace, uint64_t workspace_bytes);

/* Render a prepared batch: clear, geometry phase 1 (keys and HQ depth),
 * geometry phase 2 (HQ colours), resolve, on the context's stream with
 * launch configuration `config`; a view alone in its pass gets the
 * single-view kernels' launches between them.  Makes no other CUDA call, so
 * it can be recorded by stream capture.  Errors: PCR_ERR_ARG for a bad
 * config, or a workspace pointer this context has not prepared
 * (pcr_batch_prepare or pcr_batch_tune). */
PCR_API pcr_status pcr_batch_launch(pcr_ctx *ctx, const void *dev_workspace, int config);

/* The number of kernel launches pcr_batch_launch(config) makes for a
 * workspace this context prepared (host computation: the clear and resolve
 * kernels, the geometry phases that have passes, and the single-view
 * launches).  Errors: PCR_ERR_ARG for NULL arguments, a bad config, or a
 * workspace this context has not prepared. */
PCR_API pcr_status pcr_batch_launch_count(pcr_ctx *ctx, const void *dev_workspace, int config, int *count);

/* Time every launch configuration on the prepared batch (each rendered a few
 * times; the outputs are overwritten) and return the fastest in *config.
 * Synchronises the stream.  Errors: PCR_ERR_ARG on NULL arguments. */
PCR_API pcr_status pcr_batch_autotune(pcr_ctx *ctx, const void *dev_workspace, int *config);

/* Result of pcr_batch_tune. */
typedef struct pcr_batch_tuning {
    uint32_t l2_budget_mb;     /* framebuffer bytes one pass over a cloud may touch (64, 96 or 128 MB) */
    int32_t config;            /* launch configuration for pcr_batch_launch / pcr_batch_capture */
    uint32_t threads;          /* its threads per block (256 or 512) */
    uint32_t unroll1, unroll2; /* its points per lane in the two geometry phases (2 or 4) */
    uint32_t from_cache;       /* 1: read from cache_path, nothing was timed */
    uint32_t tried;            /* (budget, configuration) pairs timed */
    uint32_t single_colors;    /* 1: the configuration adds HQ colours with the single-view pass */
    double best_ms;            /* the winner's time per batch (0 when from the cache) */
    double default_ms;         /* pcr_batch_prepare's budget with configuration 0 (0 when from the cache) */
} pcr_batch_tuning;

/* Prepare a batch (as pcr_batch_prepare) with its tuned L2 budget, and
 * choose its launch configuration.  Tries every budget in {64, 96, 128} MB
 * with every launch configuration (threads per block x points per lane of
 * each phase x where the colours are added: 16), each timed over three launches after a warm-up, on the
 * batch's own clouds and buffers (they are rendered), and leaves the
 * workspace prepared with the fastest budget.  With cache_path (a file of
 * JSON lines, created if missing; NULL for none), a result found for this
 * GPU (name and SM count) and batch shape (cloud sizes, and each view's
 * size, flags and cloud; not its camera) is used without timing, and a new
 * result is appended.  Synchronises the context's stream.  Errors: as
 * pcr_batch_prepare; PCR_ERR_ARG for a NULL out.  A cache file that cannot
 * be read or written is ignored. */
PCR_API pcr_status pcr_batch_tune(pcr_ctx *ctx, const pcr_batch_cloud *clouds, uint32_t num_clouds,
                                  const pcr_batch_view *views, uint32_t num_views, float depth_factor,
                                  uint32_t background_rgba, void *dev_workspace, uint64_t workspace_bytes,
                                  const char *cache_path, pcr_batch_tuning *out);

/* Record pcr_batch_launch(config) into a CUDA graph and instantiate it;
 * *graph_exec receives a cudaGraphExec_t.  Launch it with pcr_graph_launch,
 * free it with pcr_graph_destroy.  Errors: PCR_ERR_ARG on NULL arguments or
 * a bad config, PCR_ERR_CUDA if capture or instantiation fails. */
PCR_API pcr_status pcr_batch_capture(pcr_ctx *ctx, const void *dev_workspace, int config, void **graph_exec);

/* Record the context's GPU work into a CUDA graph: between
 * pcr_capture_begin and pcr_capture_end, the calls that launch work (clear,
 * render, resolve, the HQ and HQS1R passes, pcr_batch_launch) are recorded
 * instead of run, with the arguments and context state of each call (buffers
 * and points are borrowed by the graph: they must outlive it).  Replaying a
 * frame then costs one launch (pcr_graph_launch) instead of one per kernel,
 * which matters for small clouds.  Calls that synchronise or copy from the
 * host (pcr_synchronize, pcr_download, pcr_upload_points_from_host,
 * pcr_last_device_error, pcr_debug_counters, pcr_check_division, the
 * reorders, pcr_batch_prepare / _tune / _autotune / _capture,
 * pcr_server_create, pcr_set_stream) return PCR_ERR_ARG while recording.
 * Errors: PCR_ERR_ARG if a capture is already open (begin) or none is (end),
 * PCR_ERR_CUDA if recording or instantiation fails (the capture is closed). */
PCR_API pcr_status pcr_capture_begin(pcr_ctx *ctx);
PCR_API pcr_status pcr_capture_end(pcr_ctx *ctx, void **graph_exec);

/* Launch an instantiated graph on the context's stream. */
PCR_API pcr_status pcr_graph_launch(pcr_ctx *ctx, void *graph_exec);

/* Destroy an instantiated graph (NULL is accepted). */
PCR_API pcr_status pcr_graph_destroy(void *graph_exec);

/* ------------------------------------------------------------------------ */
/* Serving: resident clouds, frame slots and continuous batching of view       */
/* requests on the batched renderer.  The paper renders one view per frame;   */
/* this loop is the build's own addition for many concurrent viewers.         */
/* ------------------------------------------------------------------------ */

typedef struct pcr_server pcr_server;

typedef struct pcr_server_config {
    void *dev_arena;           /* caller-owned device memory, 256-byte aligned: */
    uint64_t arena_bytes;      /*   frame slots, batch workspaces, then resident clouds */
    uint32_t max_width;        /* largest request, 1..16384 */
    uint32_t max_height;
    uint32_t num_slots;        /* frame slots: requests that can be rendering or awaiting release */
    uint32_t max_batch_views;  /* requests per batch, 1..PCR_BATCH_MAX_VIEWS */
    uint32_t max_inflight;     /* batches launched and not yet retired, 1..8 */
    uint32_t streams;          /* streams they rotate over, 1..max_inflight (0 = max_inflight):
                                  1 queues batches back to back, more lets them run concurrently */
    uint32_t max_batch_clouds; /* distinct clouds per batch, 0 = no limit: fewer clouds per batch
                                  means more views share each pass over a cloud's points */
    int32_t batch_config;      /* launch configuration of pcr_batch_launch */
    float depth_factor;        /* HQ depth band, e.g. 1.01 */
    uint32_t background_rgba;
    uint32_t max_queue;        /* admission: queued requests at most, 0 = no bound; beyond it
                                  pcr_server_submit returns PCR_ERR_BUSY */
    uint32_t deadline_us;      /* a request still queued this long after its submission expires
                                  instead of rendering (PCR_REQUEST_EXPIRED), 0 = never */
    uint32_t policy;           /* PCR_SERVE_ARRIVAL or PCR_SERVE_LARGEST_GROUP */
    uint32_t l2_budget_mb;     /* framebuffer bytes one pass over a cloud may touch, in MB (views of a
                                  cloud are packed into passes that fit); 0 = 64, at most 1024 */
} pcr_server_config;

/* Which queued requests a new batch takes (pcr_server_step). */
enum {
    PCR_SERVE_ARRIVAL = 0,       /* in arrival order, up to max_batch_clouds distinct clouds */
    PCR_SERVE_LARGEST_GROUP = 1  /* the oldest request's cloud, then the clouds with the most queued
                                    requests (up to max_batch_clouds), each cloud's requests in arrival
                                    order: more views share each pass over a cloud's points */
};

typedef struct pcr_request {
    uint32_t cloud_id;
    float matrix[16];
    int32_t width;
    int32_t height;
    uint32_t flags;            /* PCR_BATCH_BASIC and/or PCR_BATCH_HQ */
} pcr_request;

typedef struct pcr_server_result {
    int32_t width, height;
    uint32_t flags;
    uint32_t pad;
    void *keys, *image;                         /* device, in the request's frame slot */
    void *hq_depth, *hq_rg, *hq_ba, *hq_image;  /* (NULL when the flag is not set) */
    double submit_us, launch_us, done_us;       /* host steady clock, microseconds */
    uint64_t points;                            /* size of the rendered cloud */
} pcr_server_result;

typedef struct pcr_server_stats {
    uint64_t submitted, completed, batches, views_launched;
    uint64_t uploads, evictions, bytes_uploaded, points_rendered;
    uint64_t peak_queue, queued, resident_clouds, resident_bytes;
    uint64_t rejected;         /* submissions refused with PCR_ERR_BUSY */
    uint64_t expired;          /* requests that reached their deadline while queued */
    uint64_t cancelled;        /* queued requests withdrawn by pcr_server_cancel */
} pcr_server_stats;

enum {
    PCR_REQUEST_QUEUED = 0,
    PCR_REQUEST_RUNNING = 1,
    PCR_REQUEST_DONE = 2,
    PCR_REQUEST_EXPIRED = 3,
    PCR_REQUEST_CANCELLED = 4
};

/* Create a server on the context's device.  Frame slots (36 bytes per pixel
 * of max_width x max_height each) and one batch workspace per in-flight batch
 * are carved from the front of the arena; the rest holds resident clouds.
 * Creates `streams` streams, and one event and one pinned host staging area
 * per in-flight batch.  Errors: PCR_ERR_ARG for bad fields, PCR_ERR_WORKSPACE if the
 * arena cannot hold the slots and workspaces, PCR_ERR_CUDA. */
PCR_API pcr_status pcr_server_create(pcr_ctx *ctx, const pcr_server_config *cfg, pcr_server **out);

/* Wait for the server's streams, then free its host resources (NULL is
 * accepted).  The arena stays the caller's. */
PCR_API pcr_status pcr_server_destroy(pcr_server *srv);

/* Register cloud `cloud_id` with its points in host memory (pinned memory
 * makes uploads asynchronous; it must stay valid while the server lives).
 * The cloud is uploaded into the arena when a request first needs it and may
 * be evicted (least recently used, never while a batch in flight reads it)
 * to make room for another.  Errors: PCR_ERR_ARG for a duplicate id, NULL
 * points with n > 0, n >= 2^32. */
PCR_API pcr_status pcr_server_add_cloud(pcr_server *srv, uint32_t cloud_id, const void *host_points, uint64_t n);

/* Register a cloud already in device memory (caller-owned, 16-byte aligned,
 * valid while the server lives); it is never uploaded or evicted. */
PCR_API pcr_status pcr_server_add_device_cloud(pcr_server *srv, uint32_t cloud_id, const void *dev_points,
                                               uint64_t n);

/* Queue a view request; *ticket identifies it.  Time stamps use the host
 * steady clock.  Errors: PCR_ERR_ARG for an unknown cloud, a size above the
 * maxima or bad flags; PCR_ERR_WORKSPACE if the cloud can never fit;
 * PCR_ERR_BUSY when max_queue requests are already queued (admission
 * control: the caller may retry later). */
PCR_API pcr_status pcr_server_submit(pcr_server *srv, const pcr_request *req, uint64_t *ticket);

/* One turn of the serving loop, never blocking on the GPU: retire batches
 * that have finished (their requests become PCR_REQUEST_DONE), expire queued
 * requests past their deadline (PCR_REQUEST_EXPIRED, reported like finished
 * ones), then launch new batches from the queued requests (policy: in arrival
 * order, or largest groups of one cloud first) as far as in-flight batches,
 * frame slots, cloud memory and max_batch_clouds allow (a request that cannot
 * join now waits while later ones go ahead; the oldest request always joins
 * the next batch that has room).  *completed (may be NULL) counts the
 * requests this call retired or expired.  Every batch runs as
 * pcr_batch_launch does (passes over a cloud's points packed into 64 MB of
 * L2, since batches may run two at a time), so a view that shares no pass
 * with another goes through the single-view kernels (pcr_render_basic with
 * early-z, pcr_render_hq with dedup+early-z).  Every request gets exactly the
 * buffers of the request rendered alone, so a result does not depend on
 * which other requests shared its batch. */
PCR_API pcr_status pcr_server_step(pcr_server *srv, uint32_t *completed);

/* PCR_REQUEST_QUEUED, _RUNNING, _DONE, _EXPIRED or _CANCELLED for a ticket
 * not yet released. */
PCR_API pcr_status pcr_server_state(pcr_server *srv, uint64_t ticket, int *state);

/* Result of a finished request: device pointers into its frame slot (valid
 * until pcr_server_release) and its time stamps.  An expired or cancelled
 * request has NULL pointers, flags 0, points 0 and done_us at its expiry or
 * cancellation. */
PCR_API pcr_status pcr_server_get_result(pcr_server *srv, uint64_t ticket, pcr_server_result *out);

/* Report up to `capacity` tickets that finished, expired or were cancelled
 * since the previous call, in completion order; *count receives how many were
 * written. */
PCR_API pcr_status pcr_server_poll_completed(pcr_server *srv, uint64_t *tickets, uint32_t capacity, uint32_t *count);

/* Withdraw a queued request: it leaves the queue unrendered, becomes
 * PCR_REQUEST_CANCELLED and is reported like a finished one (poll, result,
 * release).  Errors: PCR_ERR_BUSY if it is already on the GPU (it will
 * finish); PCR_ERR_ARG for an unknown ticket or one already finished. */
PCR_API pcr_status pcr_server_cancel(pcr_server *srv, uint64_t ticket);

/* Give a finished request's frame slot back (or forget an expired or
 * cancelled request).
 * Reads of the slot issued on other streams must have completed first: the
 * slot may be rewritten by the next batch. */
PCR_API pcr_status pcr_server_release(pcr_server *srv, uint64_t ticket);

/* Counters since creation, plus the current queue length and residency. */
PCR_API pcr_status pcr_server_stats_get(pcr_server *srv, pcr_server_stats *out);

/* Largest cloud pcr_reorder_morton_shuffle128_noalloc accepts. */
#define PCR_REORDER_NOALLOC_MAX_POINTS 262144u

/* Allocation-free form of pcr_reorder_morton_shuffle128.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory, so cannot provide the reorder workspace.  Examples: a plugin
 * whose host application hands it only the point buffer; code running where
 * another allocator (a framework's caching pool) owns the device memory, so
 * a raw allocation would fail or fragment it; a frame loop that must not
 * stall, because allocating and freeing device memory synchronises the
 * device.
 *
 * Same orders, arguments and results as pcr_reorder_morton_shuffle128, with
 * the workspace replaced by a fixed scratch array inside the library.  The
 * array holds PCR_REORDER_NOALLOC_MAX_POINTS points' worth of workspace
 * (about 8.5 MB).  It is part of the library's device code, so every GPU that
 * loads the library holds it until the process exits.
 *   - n > PCR_REORDER_NOALLOC_MAX_POINTS: returns PCR_ERR_WORKSPACE, launches
 *     nothing.
 *   - The first call on a device looks up the array's device address, with
 *     the context's device current.  Make that first call before any stream
 *     capture.  The address stays cached for the process; creating a context
 *     (pcr_create) for the device drops it, so after a device reset
 *     (cudaDeviceReset) create a new context before calling again.
 *   - Treat the first call on a device as a warm-up.  Under lazy module
 *     loading (CUDA's default) the library's device code, this array
 *     included, is loaded onto a device only when it is first needed there,
 *     and that load takes device memory on the driver's side and may
 *     synchronise the device.  Later calls take no device memory.
 *   - All calls on a device share the one array and leave their scratch data
 *     in it.  No call needs it cleared: every scratch word a call reads, it
 *     has written first.
 *   - Calls whose work overlaps on the GPU (on different streams, or from
 *     different contexts on one device) race on the array and corrupt each
 *     other's results.  Issue them on one stream, or give each its own
 *     workspace through pcr_reorder_morton_shuffle128.
 *   - Calls no cudaMalloc, cudaFree or other allocating routine.
 * Errors: as pcr_reorder_morton_shuffle128, plus PCR_ERR_CUDA if the array's
 * address cannot be obtained. */
PCR_API pcr_status pcr_reorder_morton_shuffle128_noalloc(pcr_ctx *ctx, void *dev_points, uint64_t n, uint64_t seed,
                                                         int mode, uint32_t *dev_perm_out);

/* Check, on the device, the screen division every geometry kernel uses
 * (Sec. 3.1's projection), against the device's IEEE operations.  The
 * kernels divide both clip coordinates by w through one reciprocal per point,
 * y = RN(1/w), got from one Newton step on the hardware estimate, and correct
 * each quotient q0 = RN(c y) to RN(q0 + (c - q0 w) y) (Markstein, IBM J. Res.
 * Dev. 34(1), 1990), for w in [2^-40, 2^40); other w take the IEEE division.
 * A diagnostic: nothing on the render path calls it.
 *   - Every w bit pattern in [w_first, w_first + w_count) that lies in the
 *     window has its reciprocal compared with the IEEE reciprocal:
 *     out[0] = mismatches.
 *   - Every pair (w, c), w from that range and in the window, c = dev_c_bits[j]
 *     (device array of c_count float bit patterns) or, when dev_c_bits is
 *     NULL, c = c_first + j * c_step (bit patterns), j < c_count:
 *     out[1] = quotients that differ from IEEE c / w where
 *     2^-30 <= |c / w| <= 2^126 (out[3] = such pairs); out[2] = screen
 *     coordinates (c / w * 0.5 + 0.5) * size that differ from the ones of the
 *     IEEE quotient, counting a pair as equal when both are culled
 *     (out[4] = pairs checked).
 * Synchronises the context's stream.  The counters live in the library's
 * device code: calls must not overlap on one device.
 * Errors: PCR_ERR_ARG for a NULL ctx or out, c_count > 0 with a zero c_step
 * and no array, or size not in (0, 16384]; PCR_ERR_CUDA if a launch or copy
 * fails. */
PCR_API pcr_status pcr_check_division(pcr_ctx *ctx, uint32_t w_first, uint32_t w_count, const uint32_t *dev_c_bits,
                                      uint32_t c_first, uint32_t c_count, uint32_t c_step, float size,
                                      uint64_t out[5]);

/* Static, human-readable name of a status code. */
PCR_API const char *pcr_status_string(pcr_status status);

/* Debug builds only (libpcr_debug.so, compiled with PCR_DEBUG): read and
 * clear the counters of the single-view geometry kernels of pcr_render_basic
 * and pcr_render_hq (the HQS1R colour pass is not counted) since the last
 * call, summed over launches:
 *   out[0] key writes (Sec. 3.1-3.4 atomics, or just-set stores),
 *   out[1] HQ depth writes (Sec. 3.5),
 *   out[2] HQ colour add pairs (pcr_render_hq),
 *   out[3] early reads (Sec. 3.2) of keys and depths.
 * These show, e.g., that Sec. 3.4's deduplication sends one atomic per
 * distinct pixel per warp row.  Synchronises the stream.  Errors:
 * PCR_ERR_UNSUPPORTED in release builds; PCR_ERR_ARG for NULL arguments;
 * PCR_ERR_CUDA if the copy fails. */
PCR_API pcr_status pcr_debug_counters(pcr_ctx *ctx, uint64_t out[4]);

/* Read and clear the device-side error word of the context's device
 * (synchronises the stream): PCR_DEVICE_ERROR_KEY_RANGE when a resolve found
 * a key naming a point index outside the borrowed cloud (the pixel took the
 * background colour), PCR_DEVICE_ERROR_WAIT_TIMEOUT when a busy-loop lock
 * wait gave up, PCR_DEVICE_ERROR_BOUNDS (debug builds) when a geometry
 * kernel's bounds check dropped a point.  *code is 0 when nothing was reported.  Errors: PCR_ERR_ARG if code is NULL,
 * PCR_ERR_CUDA if the read fails. */
PCR_API pcr_status pcr_last_device_error(pcr_ctx *ctx, uint32_t *code);

#ifdef __cplusplus
}
#endif
#endif /* PCR_H */
