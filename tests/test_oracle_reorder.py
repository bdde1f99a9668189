"""Pins for the oracle's vertex-order functions (CPU only).

Morton order is checked against a depth-first octree traversal, which Sec. 5
states it is equivalent to; SplitMix64 against its published output sequence;
the shuffled orders against the properties Sec. 4 and Sec. 5 define.
"""
import numpy as np
import pytest

from conftest import read_golden
import constructed as cs
from paper_2104_07526_gb300 import scenes


def _grid_cloud(coords: np.ndarray) -> np.ndarray:
    return cs.pack(coords.astype(np.float64), np.zeros(coords.shape[0], np.uint32))


def test_morton_hand_codes(oracle):
    for row in read_golden("morton_cases.txt"):
        x, y, z, code = (int(v) for v in row[0].split())
        cloud = _grid_cloud(np.array([[0, 0, 0], [1023, 1023, 1023], [x, y, z]]))
        codes = oracle.morton_codes(cloud)
        assert codes[0] == 0
        assert codes[1] == (1 << 30) - 1
        assert codes[2] == code, (x, y, z)


def test_morton_extent_axis(oracle):
    for pts_text, codes_text in read_golden("morton_extent_cases.txt"):
        xyz = np.array([[float(v) for v in p.split()] for p in pts_text.split("|")])
        codes = oracle.morton_codes(_grid_cloud(xyz))
        assert codes.tolist() == [int(v) for v in codes_text.split()], pts_text


def _octree_dfs(points: np.ndarray, lo: np.ndarray, side: float, levels: int) -> list[int]:
    """Depth-first octree traversal with children visited x-major, then y,
    then z (lower half first); a leaf keeps its points in input order."""
    order = []

    def visit(ids, origin, h, depth):
        if depth == levels or len(ids) <= 1:
            order.extend(ids)
            return
        half = h / 2.0
        for cx in (0, 1):
            for cy in (0, 1):
                for cz in (0, 1):
                    o = origin + half * np.array([cx, cy, cz])
                    sel = [i for i in ids
                           if all((points[i, a] >= o[a]) and (points[i, a] < o[a] + half) for a in range(3))]
                    if sel:
                        visit(sel, o, half, depth + 1)

    visit(list(range(points.shape[0])), lo.astype(np.float64), side, 0)
    return order


def test_morton_equals_octree_dfs(oracle):
    """Sec. 5: sorting by Morton code equals depth-first octree traversal.
    Points sit at centres of the 1024^3 grid cells, so no point is near a
    split plane and float32 quantisation cannot move it across one."""
    rng = np.random.default_rng(11)
    cells = rng.integers(0, 1024, size=(600, 3))
    cells = np.concatenate([cells, cells[:40]])  # duplicates: ties keep input order
    cells = cells[rng.permutation(cells.shape[0])]
    lo = np.array([-3.0, 2.0, 0.5])
    side = 8.0
    xyz = lo + (cells + 0.5) * (side / 1024.0)
    # pin the bounds so the root cube is exactly [lo, lo + side)^3
    xyz = np.concatenate([[lo], [lo + side * (1023.5 / 1024.0)], xyz])
    pts = cs.pack(xyz, np.zeros(xyz.shape[0], np.uint32))
    f = np.ascontiguousarray(pts[:, :3]).view(np.float32).astype(np.float64)
    lo_f = f.min(axis=0)
    side_f = float((f.max(axis=0) - lo_f).max())
    # the oracle quantises with 1024 / extent and clamps the far corner into
    # the last cell; an octree over a cube a hair larger than the extent has
    # the same leaf cells and keeps the far corner inside
    expect = _octree_dfs(f, lo_f, side_f * (1.0 + 2.0 ** -20), 10)
    got = oracle.reorder(pts, seed=0, mode=oracle.MORTON)
    assert list(got) == expect


def test_morton63_hand_codes(oracle):
    rows = read_golden("morton63_cases.txt")
    assert len(rows) >= 10
    top = (1 << 21) - 1
    for row in rows:
        x, y, z, code = (int(v) for v in row[0].split())
        cloud = _grid_cloud(np.array([[0, 0, 0], [top, top, top], [x, y, z]]))
        codes = oracle.morton_codes63(cloud)
        assert codes[0] == 0
        assert int(codes[1]) == (1 << 63) - 1
        assert int(codes[2]) == code, (x, y, z)


def test_morton63_equals_octree_dfs(oracle):
    """Sec. 5's 21-level octree: sorting by the 63-bit code equals depth-first
    traversal.  The root cube is [0, 2^21)^3 (corner points at 0 and 2^21, so
    the scale is exactly 1) and points sit at cell centres c + 0.5, exact in
    float32; clusters of neighbouring cells and duplicates drive the
    traversal down to the last level."""
    rng = np.random.default_rng(12)
    top = 1 << 21
    cells = rng.integers(0, top, size=(300, 3))
    base = rng.integers(0, top - 8, size=(20, 3))
    cluster = np.concatenate([b + rng.integers(0, 4, size=(6, 3)) for b in base])
    cells = np.concatenate([cells, cluster, cells[:30]])
    cells = cells[rng.permutation(cells.shape[0])]
    xyz = np.concatenate([[[0.0, 0.0, 0.0]], [[float(top)] * 3], cells + 0.5])
    pts = cs.pack(xyz, np.zeros(xyz.shape[0], np.uint32))
    f = np.ascontiguousarray(pts[:, :3]).view(np.float32).astype(np.float64)
    assert np.array_equal(f, xyz)
    expect = _octree_dfs(f, np.zeros(3), float(top) * (1.0 + 2.0 ** -30), 21)
    got = oracle.reorder(pts, seed=0, mode=oracle.MORTON63)
    assert list(got) == expect


@pytest.mark.parametrize("gen", ["random", "scan"])
def test_morton63_top_bits_are_morton30(oracle, gen):
    """2^21 / e is 2^11 times 1024 / e exactly in float32, so the 21-bit cell
    of a coordinate, shifted right by 11, is its 10-bit cell (both clamp at
    the far face): the top 30 bits of the 63-bit code are the 30-bit code."""
    cloud = (scenes.random_cloud(5000, seed=4) if gen == "random" else scenes.scan(5000, seed=4)).numpy()
    c63 = oracle.morton_codes63(cloud)
    c30 = oracle.morton_codes(cloud)
    assert np.array_equal(c63 >> np.uint64(33), c30.astype(np.uint64))
    assert np.any(c63 & np.uint64((1 << 33) - 1))


def test_splitmix64_published_vector(oracle):
    for row in read_golden("splitmix64.txt"):
        seed, k, out = (int(v) for v in row[0].split())
        assert oracle.splitmix64(seed, k) == out


def test_counter_keys_match_generator(oracle):
    keys = oracle.counter_keys(1234567, 5)
    assert keys.tolist() == [oracle.splitmix64(1234567, k) >> 32 for k in range(5)]
    assert keys[0] == 6457827717110365317 >> 32


@pytest.mark.parametrize("n", [0, 1, 5, 127, 128, 129, 1000, 4097])
def test_reorder_properties(oracle, n):
    cloud = scenes.random_cloud(n, seed=n).numpy() if n else np.zeros((0, 4), np.int32)
    codes = oracle.morton_codes(cloud) if n else np.zeros(0, np.uint32)
    seed = 0x1234_5678_9ABC
    # Morton: stable sort by code
    pm = oracle.reorder(cloud, seed, oracle.MORTON)
    assert sorted(pm.tolist()) == list(range(n))
    keyed = sorted(range(n), key=lambda i: (int(codes[i]), i))
    assert pm.tolist() == keyed
    # shuffled Morton: whole 128-point batches of the Morton order, in order
    # of the high half of SplitMix64 output b, ties by batch index
    ps = oracle.reorder(cloud, seed, oracle.MORTON_SHUFFLE, 128)
    nb = (n + 127) // 128
    bkeys = [oracle.splitmix64(seed, b) >> 32 for b in range(nb)]
    border = sorted(range(nb), key=lambda b: (bkeys[b], b))
    expect = []
    for b in border:
        expect.extend(pm[b * 128:min(n, b * 128 + 128)].tolist())
    assert ps.tolist() == expect
    # shuffled: per-point high half of SplitMix64 output i
    pr = oracle.reorder(cloud, seed, oracle.SHUFFLE)
    pkeys = [oracle.splitmix64(seed, i) >> 32 for i in range(n)]
    assert pr.tolist() == sorted(range(n), key=lambda i: (pkeys[i], i))
    # the same two orders with the 63-bit code
    codes63 = oracle.morton_codes63(cloud) if n else np.zeros(0, np.uint64)
    pm63 = oracle.reorder(cloud, seed, oracle.MORTON63)
    assert pm63.tolist() == sorted(range(n), key=lambda i: (int(codes63[i]), i))
    ps63 = oracle.reorder(cloud, seed, oracle.MORTON63_SHUFFLE, 128)
    expect = []
    for b in border:
        expect.extend(pm63[b * 128:min(n, b * 128 + 128)].tolist())
    assert ps63.tolist() == expect


def test_reorder_degenerate_extent(oracle):
    """All points equal: every code is 0, so Morton order keeps input order."""
    cloud = cs.pack(np.tile([[1.5, -2.0, 3.0]], (300, 1)), np.arange(300, dtype=np.uint32))
    assert np.all(oracle.morton_codes(cloud) == 0)
    assert np.all(oracle.morton_codes63(cloud) == 0)
    assert oracle.reorder(cloud, 7, oracle.MORTON).tolist() == list(range(300))
    assert oracle.reorder(cloud, 7, oracle.MORTON63).tolist() == list(range(300))


def test_gather(oracle):
    cloud = scenes.random_cloud(257, seed=1).numpy()
    perm = oracle.reorder(cloud, 3, oracle.MORTON_SHUFFLE)
    out = oracle.gather(cloud, perm)
    assert np.array_equal(out, cloud[perm.astype(np.int64)])


def test_reorder_rejects_bad_mode(oracle):
    cloud = scenes.random_cloud(10).numpy()
    for mode in (5, 7, -1):
        with pytest.raises(ValueError):
            oracle.reorder(cloud, 0, mode)
    with pytest.raises(ValueError):
        oracle.reorder(cloud, 0, oracle.MORTON63_SHUFFLE, batch=0)
