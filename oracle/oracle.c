/*
 * CPU oracle for compute-based point rendering.  TEST INFRASTRUCTURE ONLY:
 * the test suite, the smoke check and the benchmark's CPU-baseline leg load
 * it; the CUDA library never does, and the two share no code.
 *
 * Each function restates one step of the paper (Schuetz, Kerbl, Wimmer,
 * EGSR 2021) in the plainest form: one loop over the points or pixels, no
 * blocking, no reordering beyond what the definition states.
 *
 * Pins (tests/test_oracle_pins.py, tests/test_oracle_reorder.py):
 *   oracle_project       hand-worked cases (tests/golden/project_cases.txt);
 *                        exact-geometry agreement with a float64 camera away
 *                        from pixel edges; the frustum edges a 60 degree
 *                        field of view fixes.
 *   oracle_render_basic  scenes built with known pixel and depth per point
 *                        (points on pixel-centre rays at dyadic depths);
 *                        order invariance; hand-worked ties.
 *   oracle_hq_*          same constructed scenes with depths inside and
 *                        outside the 1% band; hand-worked averages
 *                        (tests/golden/hq_cases.txt).
 *   oracle_resolve_*     hand-worked cases.
 *   oracle_*_threads     equal to the single-threaded functions on scenes
 *                        with heavy per-pixel contention.
 *   oracle_*_rgb         constructed scenes (colour of the nearest point);
 *                        hand-worked depth ties broken by colour
 *                        (tests/golden/rgb_key_cases.txt); agreement with
 *                        the index-payload render wherever the nearest
 *                        point is unique.
 *   oracle_morton_codes63 hand-worked codes (tests/golden/morton63_cases.txt);
 *                        equality of the order with a 21-level depth-first
 *                        octree traversal; its top 30 bits equal the 10-level
 *                        code (2^21 / e is 2^11 times 1024 / e exactly).
 *   oracle_morton_codes  hand-worked codes; equality of the Morton order with
 *                        a depth-first octree traversal (Sec. 5 states the
 *                        two are the same).
 *   oracle_splitmix64    the published SplitMix64 output sequence for seed
 *                        1234567.
 *   oracle_reorder       permutation, batch contiguity and batch-key order.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static float bits_to_float(uint32_t u) {
    float f;
    memcpy(&f, &u, 4);
    return f;
}

static uint32_t float_to_bits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/*
 * Sec. 3.1, Listing "basic": pos = worldViewProj * position, then
 * toPixelID(pos).  The paper leaves toPixelID undefined; the reading here:
 *   - M is row-major and clip = M (x, y, z, 1)^T, each row summed left to
 *     right: ((m0 x + m1 y) + m2 z) + m3, every product and sum rounded
 *     to float32 on its own;
 *   - w = clip.w is the linear depth (Sec. 3.1 uses pos.w directly);
 *   - the point is culled unless w > 0 and w is finite;
 *   - ndc = clip.xy / w (IEEE division), s = (ndc * 0.5 + 0.5) * size;
 *   - the point is culled unless 0 <= s < size on both axes (right and top
 *     edges exclusive); pixel = floor(sx) + floor(sy) * width, with row 0 at
 *     the bottom as in OpenGL's window coordinates.
 * There is no near or far plane test.
 */
int oracle_project(const float m[16], int width, int height, float x, float y, float z,
                   uint32_t *pixel, float *w_out) {
    float cx = ((m[0] * x + m[1] * y) + m[2] * z) + m[3];
    float cy = ((m[4] * x + m[5] * y) + m[6] * z) + m[7];
    float w = ((m[12] * x + m[13] * y) + m[14] * z) + m[15];
    if (!(w > 0.0f) || !(w < INFINITY)) return 0;
    float ndcx = cx / w;
    float ndcy = cy / w;
    float fw = (float)width;
    float fh = (float)height;
    float sx = (ndcx * 0.5f + 0.5f) * fw;
    float sy = (ndcy * 0.5f + 0.5f) * fh;
    if (!(sx >= 0.0f && sx < fw)) return 0;
    if (!(sy >= 0.0f && sy < fh)) return 0;
    uint32_t px = (uint32_t)floorf(sx);
    uint32_t py = (uint32_t)floorf(sy);
    *pixel = px + py * (uint32_t)width;
    *w_out = w;
    return 1;
}

/* Sec. 3.1: depth in the upper 32 bits, payload in the lower 32.  The payload
 * here is the point's index (its colour is looked up in the resolve), so the
 * smallest depth wins and, at equal depth, the smallest index. */
uint64_t oracle_key(float w, uint32_t index) {
    return ((uint64_t)float_to_bits(w) << 32) | (uint64_t)index;
}

void oracle_clear_keys(uint64_t *keys, size_t npx) {
    for (size_t p = 0; p < npx; ++p) keys[p] = UINT64_MAX;
}

void oracle_clear_hq(uint32_t *depth, uint64_t *rg, uint64_t *ba, size_t npx) {
    for (size_t p = 0; p < npx; ++p) {
        depth[p] = 0x7F800000u; /* +inf */
        rg[p] = 0;
        ba[p] = 0;
    }
}

/* Sec. 3.1: every visible point's key lowers its pixel's word to the minimum
 * of the two.  Order does not matter for a minimum, so a sequential loop
 * states it exactly. */
void oracle_render_basic(const oracle_point *pts, uint64_t n, const float m[16], int width, int height,
                         uint64_t *keys) {
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t p;
        float w;
        if (!oracle_project(m, width, height, pts[i].x, pts[i].y, pts[i].z, &p, &w)) continue;
        uint64_t k = oracle_key(w, (uint32_t)i);
        if (k < keys[p]) keys[p] = k;
    }
}

/* Sec. 3.5: the depth pass keeps the smallest linear depth per pixel as a
 * 32-bit value.  w > 0, so its float bits order like unsigned integers. */
void oracle_hq_depth(const oracle_point *pts, uint64_t n, const float m[16], int width, int height,
                     uint32_t *depth) {
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t p;
        float w;
        if (!oracle_project(m, width, height, pts[i].x, pts[i].y, pts[i].z, &p, &w)) continue;
        uint32_t d = float_to_bits(w);
        if (d < depth[p]) depth[p] = d;
    }
}

/* Sec. 3.5, Listing "hqs_render": a point contributes when its depth is at
 * most the stored depth times (1 + epsilon); epsilon = 1% in the paper.  The
 * threshold is the float32 product of the stored depth and depth_factor.  The
 * four 32-bit sums are packed into two 64-bit words and added as such. */
void oracle_hq_color(const oracle_point *pts, uint64_t n, const float m[16], int width, int height,
                     float depth_factor, const uint32_t *depth, uint64_t *rg, uint64_t *ba) {
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t p;
        float w;
        if (!oracle_project(m, width, height, pts[i].x, pts[i].y, pts[i].z, &p, &w)) continue;
        float limit = bits_to_float(depth[p]) * depth_factor;
        if (!(w <= limit)) continue;
        uint64_t r = pts[i].rgba & 0xFFu;
        uint64_t g = (pts[i].rgba >> 8) & 0xFFu;
        uint64_t b = (pts[i].rgba >> 16) & 0xFFu;
        rg[p] += (r << 32) | g;
        ba[p] += (b << 32) | 1u;
    }
}

void oracle_hq_channel_sums(const oracle_point *pts, uint64_t n, const float m[16], int width, int height,
                            float depth_factor, const uint32_t *depth, uint64_t *r, uint64_t *g,
                            uint64_t *b, uint64_t *count) {
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t p;
        float w;
        if (!oracle_project(m, width, height, pts[i].x, pts[i].y, pts[i].z, &p, &w)) continue;
        float limit = bits_to_float(depth[p]) * depth_factor;
        if (!(w <= limit)) continue;
        r[p] += pts[i].rgba & 0xFFu;
        g[p] += (pts[i].rgba >> 8) & 0xFFu;
        b[p] += (pts[i].rgba >> 16) & 0xFFu;
        count[p] += 1;
    }
}

/* Sec. 3.1, Listing "resolve": turn the key buffer into colours. */
void oracle_resolve_basic(const uint64_t *keys, size_t npx, const oracle_point *pts, uint64_t n,
                          uint32_t background, uint32_t *out) {
    for (size_t p = 0; p < npx; ++p) {
        uint64_t k = keys[p];
        uint64_t idx = k & 0xFFFFFFFFu;
        if (k == UINT64_MAX || idx >= n)
            out[p] = background;
        else
            out[p] = pts[idx].rgba;
    }
}

/* Sec. 3.1, Listing "basic" as printed: point = (depth << 24) | rgb, where
 * depth is the float bits of w (positive, so its bits order like the float)
 * and rgb the colour's 8 bits per channel in the 24 low bits.  The depth
 * field sits above the colour, so a minimum over keys is a minimum over
 * depth first and colour second. */
uint64_t oracle_key_rgb(float w, uint32_t rgba) {
    return ((uint64_t)float_to_bits(w) << 24) | (uint64_t)(rgba & 0xFFFFFFu);
}

void oracle_render_rgb(const oracle_point *pts, uint64_t n, const float m[16], int width, int height,
                       uint64_t *keys) {
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t p;
        float w;
        if (!oracle_project(m, width, height, pts[i].x, pts[i].y, pts[i].z, &p, &w)) continue;
        uint64_t k = oracle_key_rgb(w, pts[i].rgba);
        if (k < keys[p]) keys[p] = k;
    }
}

/* Sec. 3.1, Listing "resolve": the colour is read from the key itself. */
void oracle_resolve_rgb(const uint64_t *keys, size_t npx, uint32_t background, uint32_t *out) {
    for (size_t p = 0; p < npx; ++p) {
        if (keys[p] == UINT64_MAX)
            out[p] = background;
        else
            out[p] = (uint32_t)(keys[p] & 0xFFFFFFu) | (0xFFu << 24);
    }
}

static int thread_count(int threads) {
#ifdef _OPENMP
    return threads > 0 ? threads : omp_get_max_threads();
#else
    (void)threads;
    return 1;
#endif
}

/* Sec. 3.1 on several threads: the same per-point minimum as
 * oracle_render_basic, each update a compare-and-swap loop that retries
 * while the point's key is still smaller than the pixel's. */
int oracle_render_basic_threads(const oracle_point *pts, uint64_t n, const float m[16], int width, int height,
                                uint64_t *keys, int threads) {
    int used = thread_count(threads);
    int64_t count = (int64_t)n;
#ifdef _OPENMP
#pragma omp parallel for num_threads(used) schedule(static)
#endif
    for (int64_t i = 0; i < count; ++i) {
        uint32_t p;
        float w;
        if (!oracle_project(m, width, height, pts[i].x, pts[i].y, pts[i].z, &p, &w)) continue;
        uint64_t k = oracle_key(w, (uint32_t)i);
        uint64_t cur = __atomic_load_n(&keys[p], __ATOMIC_RELAXED);
        while (k < cur && !__atomic_compare_exchange_n(&keys[p], &cur, k, 1, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
        }
    }
    return used;
}

int oracle_resolve_basic_threads(const uint64_t *keys, size_t npx, const oracle_point *pts, uint64_t n,
                                 uint32_t background, uint32_t *out, int threads) {
    int used = thread_count(threads);
    int64_t count = (int64_t)npx;
#ifdef _OPENMP
#pragma omp parallel for num_threads(used) schedule(static)
#endif
    for (int64_t p = 0; p < count; ++p) {
        uint64_t k = keys[p];
        uint64_t idx = k & 0xFFFFFFFFu;
        out[p] = (k == UINT64_MAX || idx >= n) ? background : pts[idx].rgba;
    }
    return used;
}

/* Sec. 3.5, Listing "hqs_resolve": divide the colour sums by the count with
 * truncating integer division.  A channel above 255 (possible only after a
 * 32-bit sum overflowed) is clamped to 255. */
void oracle_resolve_hq(const uint64_t *rg, const uint64_t *ba, size_t npx, uint32_t background,
                       uint32_t *out) {
    for (size_t p = 0; p < npx; ++p) {
        uint32_t a = (uint32_t)(ba[p] & 0xFFFFFFFFu);
        if (a == 0) {
            out[p] = background;
            continue;
        }
        uint32_t r = (uint32_t)(rg[p] >> 32) / a;
        uint32_t g = (uint32_t)(rg[p] & 0xFFFFFFFFu) / a;
        uint32_t b = (uint32_t)(ba[p] >> 32) / a;
        if (r > 255) r = 255;
        if (g > 255) g = 255;
        if (b > 255) b = 255;
        out[p] = r | (g << 8) | (b << 16) | (0xFFu << 24);
    }
}

/* ------------------------------------------------------------------------ */
/* Vertex order (Sec. 4, Sec. 5 list of orderings)                           */
/* ------------------------------------------------------------------------ */

void oracle_aabb(const oracle_point *pts, uint64_t n, float lo[3], float hi[3]) {
    for (int a = 0; a < 3; ++a) {
        lo[a] = INFINITY;
        hi[a] = -INFINITY;
    }
    for (uint64_t i = 0; i < n; ++i) {
        float v[3] = {pts[i].x, pts[i].y, pts[i].z};
        for (int a = 0; a < 3; ++a) {
            if (v[a] < lo[a]) lo[a] = v[a];
            if (v[a] > hi[a]) hi[a] = v[a];
        }
    }
}

/* Quantise one coordinate to 10 bits: floor((v - lo) * scale), clamped to
 * [0, 1023]; NaN maps to 0. */
static uint32_t quantise10(float v, float lo, float scale) {
    float f = floorf((v - lo) * scale);
    if (!(f >= 0.0f)) return 0;
    if (f >= 1023.0f) return 1023;
    return (uint32_t)f;
}

/* Sec. 5: sort by Morton code, i.e. depth-first order of an octree.  The
 * paper uses 21 levels; this build uses 10 levels (a 30-bit code).  The
 * octree's root cell is the cube with the bounds' minimum corner and the
 * largest extent as side; a zero or non-finite extent gives every point
 * code 0. */
void oracle_morton_codes(const oracle_point *pts, uint64_t n, uint32_t *codes) {
    float lo[3], hi[3];
    oracle_aabb(pts, n, lo, hi);
    float ext = hi[0] - lo[0];
    float ey = hi[1] - lo[1];
    float ez = hi[2] - lo[2];
    if (ey > ext) ext = ey;
    if (ez > ext) ext = ez;
    int degenerate = !(ext > 0.0f) || !(ext < INFINITY);
    float scale = degenerate ? 0.0f : 1024.0f / ext;
    for (uint64_t i = 0; i < n; ++i) {
        if (degenerate) {
            codes[i] = 0;
            continue;
        }
        uint32_t q[3] = {quantise10(pts[i].x, lo[0], scale), quantise10(pts[i].y, lo[1], scale),
                         quantise10(pts[i].z, lo[2], scale)};
        uint32_t c = 0;
        for (int bit = 0; bit < 10; ++bit) {
            c |= ((q[0] >> bit) & 1u) << (3 * bit + 2);
            c |= ((q[1] >> bit) & 1u) << (3 * bit + 1);
            c |= ((q[2] >> bit) & 1u) << (3 * bit);
        }
        codes[i] = c;
    }
}

/* Quantise one coordinate to 21 bits: floor((v - lo) * scale), clamped to
 * [0, 2^21 - 1]; NaN maps to 0. */
static uint32_t quantise21(float v, float lo, float scale) {
    float f = floorf((v - lo) * scale);
    if (!(f >= 0.0f)) return 0;
    if (f >= 2097151.0f) return 2097151u;
    return (uint32_t)f;
}

/* Sec. 5: the paper's 21-level octree, as a 63-bit code.  Same root cube and
 * degenerate case as oracle_morton_codes, with 2^21 cells per axis. */
void oracle_morton_codes63(const oracle_point *pts, uint64_t n, uint64_t *codes) {
    float lo[3], hi[3];
    oracle_aabb(pts, n, lo, hi);
    float ext = hi[0] - lo[0];
    float ey = hi[1] - lo[1];
    float ez = hi[2] - lo[2];
    if (ey > ext) ext = ey;
    if (ez > ext) ext = ez;
    int degenerate = !(ext > 0.0f) || !(ext < INFINITY);
    float scale = degenerate ? 0.0f : 2097152.0f / ext;
    for (uint64_t i = 0; i < n; ++i) {
        if (degenerate) {
            codes[i] = 0;
            continue;
        }
        uint32_t q[3] = {quantise21(pts[i].x, lo[0], scale), quantise21(pts[i].y, lo[1], scale),
                         quantise21(pts[i].z, lo[2], scale)};
        uint64_t c = 0;
        for (int bit = 0; bit < 21; ++bit) {
            c |= (uint64_t)((q[0] >> bit) & 1u) << (3 * bit + 2);
            c |= (uint64_t)((q[1] >> bit) & 1u) << (3 * bit + 1);
            c |= (uint64_t)((q[2] >> bit) & 1u) << (3 * bit);
        }
        codes[i] = c;
    }
}

/* SplitMix64 as published: state advances by the golden-ratio increment and
 * each output is the mixed state.  Output k uses state seed + (k + 1) * gamma. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void oracle_counter_keys(uint64_t seed, uint64_t count, uint32_t *keys) {
    for (uint64_t k = 0; k < count; ++k) keys[k] = (uint32_t)(oracle_splitmix64(seed, k) >> 32);
}

typedef struct {
    uint32_t key;
    uint32_t index;
} keyed;

/* Stable sort by key == sort by (key, original position). */
static int keyed_cmp(const void *a, const void *b) {
    const keyed *x = (const keyed *)a, *y = (const keyed *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->index != y->index) return x->index < y->index ? -1 : 1;
    return 0;
}

typedef struct {
    uint64_t key;
    uint32_t index;
} keyed64;

static int keyed64_cmp(const void *a, const void *b) {
    const keyed64 *x = (const keyed64 *)a, *y = (const keyed64 *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->index != y->index) return x->index < y->index ? -1 : 1;
    return 0;
}

/* perm = the points in stable order of their Morton code (the 30-bit code,
 * or the 63-bit one when wide).  Returns 0, or -1 when allocation fails. */
static int morton_order(const oracle_point *pts, uint64_t n, int wide, uint32_t *perm) {
    keyed64 *k = (keyed64 *)malloc(n * sizeof(keyed64));
    uint64_t *codes = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint32_t *narrow = wide ? NULL : (uint32_t *)malloc(n * sizeof(uint32_t));
    if (!k || !codes || (!wide && !narrow)) {
        free(k);
        free(codes);
        free(narrow);
        return -1;
    }
    if (wide) {
        oracle_morton_codes63(pts, n, codes);
    } else {
        oracle_morton_codes(pts, n, narrow);
        for (uint64_t i = 0; i < n; ++i) codes[i] = narrow[i];
    }
    for (uint64_t i = 0; i < n; ++i) {
        k[i].key = codes[i];
        k[i].index = (uint32_t)i;
    }
    qsort(k, n, sizeof(keyed64), keyed64_cmp);
    for (uint64_t i = 0; i < n; ++i) perm[i] = k[i].index;
    free(narrow);
    free(codes);
    free(k);
    return 0;
}

int oracle_reorder(const oracle_point *pts, uint64_t n, uint64_t seed, int mode, uint32_t batch,
                   uint32_t *perm) {
    if (n > 0xFFFFFFFFull || mode < 0 || mode > 4 || ((mode == 1 || mode == 4) && batch == 0)) return -1;
    if (n == 0) return 0;
    if (mode == 2) {
        /* Sec. 5, "Shuffled": a random value per point, then sort by it. */
        keyed *k = (keyed *)malloc(n * sizeof(keyed));
        if (!k) return -1;
        for (uint64_t i = 0; i < n; ++i) {
            k[i].key = (uint32_t)(oracle_splitmix64(seed, i) >> 32);
            k[i].index = (uint32_t)i;
        }
        qsort(k, n, sizeof(keyed), keyed_cmp);
        for (uint64_t i = 0; i < n; ++i) perm[i] = k[i].index;
        free(k);
        return 0;
    }
    const int wide = mode >= 3;
    if (mode == 0 || mode == 3) return morton_order(pts, n, wide, perm);
    uint32_t *morton = (uint32_t *)malloc(n * sizeof(uint32_t));
    if (!morton) return -1;
    if (morton_order(pts, n, wide, morton) != 0) {
        free(morton);
        return -1;
    }
    /* Sec. 4 and Sec. 5, "Shuffled Morton": cut the Morton order into batches
     * of `batch` points (the last one may be shorter), move whole batches to
     * random positions, keep each batch's inner order. */
    uint64_t nb = (n + batch - 1) / batch;
    keyed *bk = (keyed *)malloc(nb * sizeof(keyed));
    if (!bk) {
        free(morton);
        return -1;
    }
    for (uint64_t b = 0; b < nb; ++b) {
        bk[b].key = (uint32_t)(oracle_splitmix64(seed, b) >> 32);
        bk[b].index = (uint32_t)b;
    }
    qsort(bk, nb, sizeof(keyed), keyed_cmp);
    uint64_t out = 0;
    for (uint64_t t = 0; t < nb; ++t) {
        uint64_t b = bk[t].index;
        uint64_t first = b * batch;
        uint64_t last = first + batch < n ? first + batch : n;
        for (uint64_t j = first; j < last; ++j) perm[out++] = morton[j];
    }
    free(bk);
    free(morton);
    return 0;
}

void oracle_gather(const oracle_point *pts, uint64_t n, const uint32_t *perm, oracle_point *out) {
    for (uint64_t j = 0; j < n; ++j) out[j] = pts[perm[j]];
}
