/*
 * CPU oracle for compute-based point rendering (Schuetz, Kerbl, Wimmer,
 * "Rendering Point Clouds with Compute Shaders and Vertex Order
 * Optimization", EGSR 2021).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded statement
 * of what the renderer computes.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * constant with the CUDA library, and the library never calls it.
 *
 * Arithmetic: float32 in a fixed operation order.  Build with
 * -ffp-contract=off and without fast-math, so every product and sum is
 * rounded on its own (no fused multiply-add).
 *
 * Point record: 16 bytes, float x, y, z, then uint32 rgba with r in the low
 * byte (Sec. 5: 796M points take 12.7 GB).
 */
#ifndef PCR_ORACLE_H
#define PCR_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oracle_point {
    float x, y, z;
    uint32_t rgba;
} oracle_point;

/* Sec. 3.1: project one point and find its pixel.  Returns 1 and writes the
 * pixel id and the linear depth w when the point is visible; returns 0 when it
 * is culled. */
int oracle_project(const float m[16], int width, int height, float x, float y, float z,
                   uint32_t *pixel, float *w);

/* Sec. 3.1: the 64-bit key (depth bits << 32 | point index). */
uint64_t oracle_key(float w, uint32_t index);

/* Clear values: keys to all ones, HQ depth to +inf bits, HQ sums to zero. */
void oracle_clear_keys(uint64_t *keys, size_t npx);
void oracle_clear_hq(uint32_t *depth, uint64_t *rg, uint64_t *ba, size_t npx);

/* Sec. 3.1: keys[p] = min(keys[p], key of every visible point landing on p).
 * Accumulates into keys; the caller clears first for a fresh frame. */
void oracle_render_basic(const oracle_point *pts, uint64_t n, const float m[16], int width, int height,
                         uint64_t *keys);

/* Sec. 3.5, depth pass: depth[p] = min(depth[p], float bits of w). */
void oracle_hq_depth(const oracle_point *pts, uint64_t n, const float m[16], int width, int height,
                     uint32_t *depth);

/* Sec. 3.5, colour pass: every visible point with w <= depth[p] * depth_factor
 * (float32 product) adds (r << 32 | g) to rg[p] and (b << 32 | 1) to ba[p],
 * modulo 2^64. */
void oracle_hq_color(const oracle_point *pts, uint64_t n, const float m[16], int width, int height,
                     float depth_factor, const uint32_t *depth, uint64_t *rg, uint64_t *ba);

/* Unpacked per-channel sums of the colour pass, in 64 bits each, so tests can
 * tell whether a packed 32-bit channel overflowed. */
void oracle_hq_channel_sums(const oracle_point *pts, uint64_t n, const float m[16], int width, int height,
                            float depth_factor, const uint32_t *depth, uint64_t *r, uint64_t *g,
                            uint64_t *b, uint64_t *count);

/* Sec. 3.1, resolve: background where the key is all ones (or names no point
 * of this cloud), else the rgba word of the point the key names. */
void oracle_resolve_basic(const uint64_t *keys, size_t npx, const oracle_point *pts, uint64_t n,
                          uint32_t background, uint32_t *out);

/* Sec. 3.1, the key as Listing "basic" prints it: depth bits shifted left
 * by 24 over a 24-bit colour payload (the rgba word's low three bytes).  The
 * smallest depth wins and, at equal depth, the smallest 24-bit colour. */
uint64_t oracle_key_rgb(float w, uint32_t rgba);

/* Sec. 3.1 with the colour payload: keys[p] = min(keys[p], oracle_key_rgb of
 * every visible point landing on p).  Accumulates like oracle_render_basic. */
void oracle_render_rgb(const oracle_point *pts, uint64_t n, const float m[16], int width, int height,
                       uint64_t *keys);

/* Sec. 3.1, resolve of colour-payload keys: background where the key is all
 * ones, else the key's 24-bit colour with alpha 255. */
void oracle_resolve_rgb(const uint64_t *keys, size_t npx, uint32_t background, uint32_t *out);

/* oracle_render_basic and oracle_resolve_basic on `threads` host threads
 * (every available one when threads <= 0; one when the oracle was built
 * without OpenMP).  Each point takes its pixel's minimum with a
 * compare-and-swap loop; a minimum does not depend on order, so the keys
 * equal oracle_render_basic's.  Used to time the oracle on all host cores.
 * Return the number of threads used. */
int oracle_render_basic_threads(const oracle_point *pts, uint64_t n, const float m[16], int width, int height,
                                uint64_t *keys, int threads);
int oracle_resolve_basic_threads(const uint64_t *keys, size_t npx, const oracle_point *pts, uint64_t n,
                                 uint32_t background, uint32_t *out, int threads);

/* Sec. 3.5, resolve: truncating integer average per channel, alpha 255;
 * background where no point contributed. */
void oracle_resolve_hq(const uint64_t *rg, const uint64_t *ba, size_t npx, uint32_t background,
                       uint32_t *out);

/* Sec. 5 ("Morton" order): axis-aligned bounds, ignoring NaN coordinates. */
void oracle_aabb(const oracle_point *pts, uint64_t n, float lo[3], float hi[3]);

/* 30-bit Morton code per point: 10 bits per axis over the cube spanned by the
 * largest extent of the bounds; x in bit 3i+2, y in bit 3i+1, z in bit 3i. */
void oracle_morton_codes(const oracle_point *pts, uint64_t n, uint32_t *codes);

/* 63-bit Morton code per point, the paper's 21 levels (Sec. 5 "Morton"): 21
 * bits per axis over the same cube as oracle_morton_codes; x in bit 3i+2, y
 * in bit 3i+1, z in bit 3i. */
void oracle_morton_codes63(const oracle_point *pts, uint64_t n, uint64_t *codes);

/* SplitMix64 (Steele, Lea, Flood 2014): the k-th output (k from 0) of the
 * generator seeded with `seed`. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t k);

/* keys[k] = high 32 bits of oracle_splitmix64(seed, k), k < count: the
 * batch (or point) keys of the shuffled orders. */
void oracle_counter_keys(uint64_t seed, uint64_t count, uint32_t *keys);

/* Sec. 4 and Sec. 5 vertex orders.  perm[new] = old.
 * mode 0: Morton order (stable sort by code).
 * mode 1: shuffled Morton: Morton order cut into batches of `batch` points,
 *         batches stably sorted by the high 32 bits of SplitMix64 output b,
 *         each batch keeps its inner order.
 * mode 2: shuffled: points stably sorted by the high 32 bits of SplitMix64
 *         output i.
 * mode 3: Morton order by the 63-bit code (stable sort).
 * mode 4: shuffled Morton over the mode 3 order (batches as in mode 1).
 * Returns 0 on success, -1 on a bad argument or allocation failure. */
int oracle_reorder(const oracle_point *pts, uint64_t n, uint64_t seed, int mode, uint32_t batch,
                   uint32_t *perm);

/* out[j] = pts[perm[j]]. */
void oracle_gather(const oracle_point *pts, uint64_t n, const uint32_t *perm, oracle_point *out);

#ifdef __cplusplus
}
#endif
#endif
