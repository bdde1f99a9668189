"""Pins for the CPU oracle's rendering functions (CPU only).

Each test checks the oracle against something other than itself: values
worked by hand from the paper's definitions (tests/golden), scenes whose
answer is known by construction, exact float64 geometry, the frustum a
60-degree field of view fixes, and invariants the paper states.
"""
import math

import numpy as np
import pytest

from conftest import read_golden
import constructed as cs
from paper_2104_07526_gb300 import scenes


def _mat(text):
    return np.array([float(v) for v in text.split()], dtype=np.float32)


# --- Sec. 3.1 projection ----------------------------------------------------

def test_project_hand_cases(oracle):
    rows = read_golden("project_cases.txt")
    assert len(rows) >= 12
    for name, m, wh, xyz, expect in rows:
        W, H = (int(v) for v in wh.split())
        x, y, z = (float(v) for v in xyz.split())
        got = oracle.project(_mat(m), W, H, x, y, z)
        if expect == "cull":
            assert got is None, name
        else:
            pix, w = expect.split()
            assert got is not None, name
            assert got[0] == int(pix), name
            assert got[1] == np.float32(float(w)), name


def test_key_hand_cases(oracle):
    for row in read_golden("key_cases.txt"):
        w, idx, expect = row[0].split()
        assert oracle.key(float(w), int(idx)) == int(expect, 16)


def test_constructed_depth_scene(oracle):
    """Points on pixel-centre rays at exact depths: the key buffer must hold,
    per pixel, the smallest depth and at a tie the smallest index."""
    rng = np.random.default_rng(1)
    cloud, expected, _, _ = cs.depth_scene(rng)
    keys = oracle.render_basic(cloud, cs.camera(), cs.W, cs.H)
    assert np.array_equal(keys, expected)


def test_frustum_edges(oracle):
    """A 60-degree vertical field of view puts the top and bottom frustum
    planes at |y| = tan(30 deg) * depth; the side planes scale by W/H."""
    m = cs.camera()
    t = math.tan(math.radians(30.0))
    for d in (1.0, 2.5, 7.0):
        z = cs.EYE_Z - d
        in_top = oracle.project(m, cs.W, cs.H, 0.0, t * d * (1 - 1e-4), z)
        assert in_top is not None and in_top[0] // cs.W == cs.H - 1
        in_bottom = oracle.project(m, cs.W, cs.H, 0.0, -t * d * (1 - 1e-4), z)
        assert in_bottom is not None and in_bottom[0] // cs.W == 0
        assert oracle.project(m, cs.W, cs.H, 0.0, t * d * (1 + 1e-4), z) is None
        assert oracle.project(m, cs.W, cs.H, 0.0, -t * d * (1 + 1e-4), z) is None
        xe = t * d * cs.W / cs.H
        right = oracle.project(m, cs.W, cs.H, xe * (1 - 1e-4), 0.0, z)
        assert right is not None and right[0] % cs.W == cs.W - 1
        left = oracle.project(m, cs.W, cs.H, -xe * (1 - 1e-4), 0.0, z)
        assert left is not None and left[0] % cs.W == 0
        assert oracle.project(m, cs.W, cs.H, xe * (1 + 1e-4), 0.0, z) is None
        # the centre of the view is the centre pixel, at depth d
        c = oracle.project(m, cs.W, cs.H, 0.0, 0.0, z)
        assert c == (cs.W // 2 + (cs.H // 2) * cs.W, np.float32(d))
    # behind the eye
    assert oracle.project(m, cs.W, cs.H, 0.0, 0.0, cs.EYE_Z + 1.0) is None


def test_exact_geometry_agreement(oracle):
    """Away from pixel edges the float32 pixel equals the pixel of the exact
    projection; w is within a few float32 ulps of the exact depth."""
    rng = np.random.default_rng(2)
    views = scenes.boxes_views() + scenes.sphere_plane_views()
    for view in views:
        m = view.matrix.astype(np.float64)
        pts = rng.uniform(-60, 60, size=(3000, 3)).astype(np.float32)
        checked = 0
        for x, y, z in pts:
            v = np.array([x, y, z, 1.0], dtype=np.float64)
            c = m @ v
            got = oracle.project(view.matrix, view.width, view.height, float(x), float(y), float(z))
            if c[3] <= 1e-6:
                assert got is None
                continue
            sx = (c[0] / c[3] * 0.5 + 0.5) * view.width
            sy = (c[1] / c[3] * 0.5 + 0.5) * view.height
            margin = 1e-3
            near_edge = min(abs(sx - round(sx)), abs(sy - round(sy))) < margin
            if near_edge:
                continue
            inside = 0 <= sx < view.width and 0 <= sy < view.height
            if not inside:
                assert got is None
                continue
            assert got is not None
            assert got[0] == int(math.floor(sx)) + int(math.floor(sy)) * view.width
            assert abs(got[1] - c[3]) <= 4 * np.spacing(np.float32(c[3]))
            checked += 1
        assert checked > 100


def test_basic_hand_ties(oracle):
    """Sec. 3.1: atomicMin keeps the smaller depth; with the index payload an
    equal depth keeps the smaller index."""
    m = _mat("1 0 0 0  0 1 0 0  0 0 1 0  0 0 1 0")  # w = z
    xyz = np.array([[0, 0, 1.0], [0, 0, 0.5], [0, 0, 0.5], [0, 0, 2.0]])
    cloud = cs.pack(xyz, cs.rgba_word([1, 2, 3, 4], 0, 0))
    keys = oracle.render_basic(cloud, m, 4, 4)
    assert keys[10] == (0x3F000000 << 32) | 1
    others = np.delete(keys, 10)
    assert np.all(others == np.uint64(0xFFFFFFFFFFFFFFFF))


def test_order_invariance(oracle):
    """Sec. 3.2 and 4: any vertex order gives the same image.  Depth halves
    must match exactly; where a pixel's minimum depth is unique the index
    halves map back through the permutation."""
    rng = np.random.default_rng(3)
    cloud = scenes.random_cloud(20000, seed=5).numpy()
    m = scenes.camera((0.3, -2.5, 2.0), (0, 0, 0), (0, 0, 1), 64, 48)
    perm = rng.permutation(cloud.shape[0])
    k0 = oracle.render_basic(cloud, m, 64, 48)
    k1 = oracle.render_basic(cloud[perm], m, 64, 48)
    assert np.array_equal(k0 >> np.uint64(32), k1 >> np.uint64(32))
    # unique minima: count points per (pixel, depth)
    hit = k0 != np.uint64(0xFFFFFFFFFFFFFFFF)
    assert hit.sum() > 500
    idx0 = (k0 & np.uint64(0xFFFFFFFF)).astype(np.int64)
    idx1 = (k1 & np.uint64(0xFFFFFFFF)).astype(np.int64)
    w = np.ascontiguousarray(cloud[:, :3]).view(np.float32)
    same = 0
    for p in np.nonzero(hit)[0]:
        if perm[idx1[p]] == idx0[p]:
            same += 1
    assert same == hit.sum()  # continuous random depths: minima are unique


def test_numpy_float32_consistency(oracle):
    """Consistency check (not a pin): a vectorised numpy float32 statement of
    the same reading agrees on a tiny cloud, ruling out indexing slips in
    the C loop."""
    cloud = scenes.random_cloud(4096, seed=9).numpy()
    W, H = 16, 12
    m = scenes.camera((0.5, -3.0, 1.5), (0, 0, 0), (0, 0, 1), W, H)
    p = np.ascontiguousarray(cloud[:, :3]).view(np.float32)
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    f = np.float32
    cx = ((m[0, 0] * x + m[0, 1] * y) + m[0, 2] * z) + m[0, 3]
    cy = ((m[1, 0] * x + m[1, 1] * y) + m[1, 2] * z) + m[1, 3]
    w = ((m[3, 0] * x + m[3, 1] * y) + m[3, 2] * z) + m[3, 3]
    with np.errstate(all="ignore"):
        sx = (cx / w * f(0.5) + f(0.5)) * f(W)
        sy = (cy / w * f(0.5) + f(0.5)) * f(H)
    ok = (w > 0) & np.isfinite(w) & (sx >= 0) & (sx < W) & (sy >= 0) & (sy < H)
    expect = np.full(W * H, np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)
    pix = np.floor(sx[ok]).astype(np.int64) + np.floor(sy[ok]).astype(np.int64) * W
    keys = (w[ok].view(np.uint32).astype(np.uint64) << np.uint64(32)) | np.nonzero(ok)[0].astype(np.uint64)
    np.minimum.at(expect, pix, keys)
    got = oracle.render_basic(cloud, m, W, H)
    assert ok.sum() > 100
    assert np.array_equal(got, expect)


# --- Sec. 3.5 high quality ----------------------------------------------------

def test_hq_hand_cases(oracle):
    m = _mat("1 0 0 0  0 1 0 0  0 0 1 0  0 0 1 0")
    for name, pts_text, sums_text, rgba_hex in read_golden("hq_cases.txt"):
        recs = [[float(v) for v in p.split()] for p in pts_text.split("|")]
        xyz = np.array([[0.0, 0.0, r[0]] for r in recs])
        rgba = cs.rgba_word([int(r[1]) for r in recs], [int(r[2]) for r in recs], [int(r[3]) for r in recs])
        cloud = cs.pack(xyz, rgba)
        d, rg, ba = oracle.render_hq(cloud, m, 4, 4, 1.01)
        er, eg, eb, ec = (int(v) for v in sums_text.split())
        assert d[10] == min(np.float32(r[0]).view(np.uint32) for r in recs), name
        assert int(rg[10]) == (er << 32) | eg, name
        assert int(ba[10]) == (eb << 32) | ec, name
        out = oracle.resolve_hq(rg, ba, 0x11223344)
        assert out[10] == int(rgba_hex, 16), name
        assert np.all(np.delete(out, 10) == 0x11223344), name


def test_hq_constructed_scene(oracle):
    rng = np.random.default_rng(4)
    cloud, depth, sums = cs.hq_scene(rng)
    m = cs.camera()
    d, rg, ba = oracle.render_hq(cloud, m, cs.W, cs.H, 1.01)
    assert np.array_equal(d, depth)
    assert np.array_equal(rg, (sums[0] << np.uint64(32)) | sums[1])
    assert np.array_equal(ba, (sums[2] << np.uint64(32)) | sums[3])
    r, g, b, c = oracle.hq_channel_sums(cloud, m, cs.W, cs.H, d, 1.01)
    assert np.array_equal(np.stack([r, g, b, c]), sums)


def test_hq_depth_factor_one_counts_only_front(oracle):
    """With a factor of exactly 1 only points at the front depth count."""
    rng = np.random.default_rng(5)
    cloud, depth, _ = cs.hq_scene(rng, npix=50)
    m = cs.camera()
    d, rg, ba = oracle.render_hq(cloud, m, cs.W, cs.H, 1.0)
    p = np.ascontiguousarray(cloud[:, :3]).view(np.float32)
    counts = np.zeros(cs.W * cs.H, dtype=np.uint64)
    for i in range(cloud.shape[0]):
        pr = oracle.project(m, cs.W, cs.H, *p[i])
        if pr and np.float32(pr[1]).view(np.uint32) == d[pr[0]]:
            counts[pr[0]] += 1
    assert np.array_equal(ba & np.uint64(0xFFFFFFFF), counts)


# --- Sec. 3.1 colour-payload key (Listing "basic" as printed) -------------------

def test_rgb_key_hand_cases(oracle):
    rows = read_golden("rgb_key_cases.txt")
    assert len(rows) >= 4
    for row in rows:
        w, rgba, expect = row[0].split()
        assert oracle.key_rgb(float(w), int(rgba, 16)) == int(expect, 16), row


def test_rgb_hand_ties(oracle):
    """An equal depth keeps the smaller 24-bit colour, whatever the index or
    the alpha byte; the index payload would keep the first of the tie."""
    m = _mat("1 0 0 0  0 1 0 0  0 0 1 0  0 0 1 0")  # w = z
    xyz = np.array([[0, 0, 1.0], [0, 0, 0.5], [0, 0, 0.5], [0, 0, 2.0], [0, 0, 0.5]])
    rgba = np.array([0xFF000010, 0xFF0000FF, 0x00000001, 0xFF000000, 0x7F000001], dtype=np.uint32)
    cloud = cs.pack(xyz, rgba)
    keys = oracle.render_rgb(cloud, m, 4, 4)
    assert keys[10] == (0x3F000000 << 24) | 0x000001
    assert np.all(np.delete(keys, 10) == np.uint64(0xFFFFFFFFFFFFFFFF))
    out = oracle.resolve_rgb(keys, background=0x11223344)
    assert out[10] == 0xFF000001 and np.all(np.delete(out, 10) == 0x11223344)
    assert oracle.resolve_basic(oracle.render_basic(cloud, m, 4, 4), cloud)[10] == 0xFF0000FF


def test_rgb_constructed_depth_scene(oracle):
    """Points on pixel-centre rays at exact depths: per pixel the smallest
    depth, at a tie the smallest colour."""
    rng = np.random.default_rng(5)
    cloud, _, recs, colour = cs.depth_scene(rng)
    expected = np.full(cs.W * cs.H, np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)
    for i, (p, _, _, d) in enumerate(recs):
        rgb = int(colour[i, 0]) | (int(colour[i, 1]) << 8) | (int(colour[i, 2]) << 16)
        key = (int(np.float32(d).view(np.uint32)) << 24) | rgb
        expected[p] = min(int(expected[p]), key)
    keys = oracle.render_rgb(cloud, cs.camera(), cs.W, cs.H)
    assert np.array_equal(keys, expected)


def test_rgb_agrees_with_index_payload(oracle):
    """Both payloads keep the same depth everywhere; where a pixel's nearest
    point is unique they name the same point, so the colours agree."""
    cloud = scenes.sphere_plane(40_000, seed=9).numpy()
    m = scenes.camera((0, 0, 4), (0, 0, 0), (0, 1, 0), 160, 120)
    k_idx = oracle.render_basic(cloud, m, 160, 120)
    k_rgb = oracle.render_rgb(cloud, m, 160, 120)
    empty = k_idx == np.uint64(0xFFFFFFFFFFFFFFFF)
    assert np.array_equal(empty, k_rgb == np.uint64(0xFFFFFFFFFFFFFFFF))
    assert np.array_equal(k_idx[~empty] >> np.uint64(32), k_rgb[~empty] >> np.uint64(24))
    depth_of = {}
    for i in range(cloud.shape[0]):
        hit = oracle.project(m, 160, 120, *cloud[i, :3].view(np.float32).tolist())
        if hit is not None:
            depth_of.setdefault(hit[0], []).append(np.float32(hit[1]).view(np.uint32))
    unique = [p for p, ds in depth_of.items() if ds.count(min(ds)) == 1]
    assert len(unique) > 1000
    c_idx = oracle.resolve_basic(k_idx, cloud)
    c_rgb = oracle.resolve_rgb(k_rgb)
    for p in unique:
        assert c_rgb[p] == (int(c_idx[p]) & 0xFFFFFF) | 0xFF000000


# --- multi-threaded timing variant ------------------------------------------------

@pytest.mark.parametrize("threads", [1, 3, 0])
def test_threads_variant_equals_single_thread(oracle, threads):
    """The host-parallel render and resolve (used only to time the oracle on
    all host cores) give exactly the single-threaded results, also when all
    points fight over one pixel."""
    sphere = scenes.sphere_plane(60_000, seed=3).numpy()
    n = 40_000
    one_px = cs.pack(np.tile([[0.0, 0.0, 1.5]], (n, 1)), np.arange(n, dtype=np.uint32))
    d = np.random.default_rng(4).integers(4, 4000, size=n) / 256.0
    one_px_depths = cs.pack(np.stack([np.zeros(n), np.zeros(n), cs.EYE_Z - d], 1), np.arange(n, dtype=np.uint32))
    for cloud in (sphere, one_px, one_px_depths):
        m = cs.camera()
        want = oracle.render_basic(cloud, m, cs.W, cs.H)
        got, used = oracle.render_basic_threads(cloud, m, cs.W, cs.H, threads)
        assert used >= 1
        assert np.array_equal(got, want)
        img, _ = oracle.resolve_basic_threads(got, cloud, 0x01020304, threads)
        assert np.array_equal(img, oracle.resolve_basic(want, cloud, 0x01020304))


# --- resolve -------------------------------------------------------------------

def test_resolve_basic_cases(oracle):
    cloud = cs.pack(np.zeros((3, 3)), np.array([0x01020304, 0xAABBCCDD, 0xFF0000FF], dtype=np.uint32))
    keys = np.array([0xFFFFFFFFFFFFFFFF, (0x3F800000 << 32) | 1, (0x3F800000 << 32) | 2,
                     (0x3F800000 << 32) | 3, 0], dtype=np.uint64)
    out = oracle.resolve_basic(keys, cloud, background=0x00000000)
    assert list(out) == [0, 0xAABBCCDD, 0xFF0000FF, 0, 0x01020304]
