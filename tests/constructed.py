"""Scenes whose expected render is known by construction (test inputs).

Every point is placed on the ray through a pixel centre of a known camera, at
a dyadic depth d.  With the camera at (0, 0, 4) looking down -z, the clip w
row of its matrix is exactly (0, 0, -1, 4), so a point at z = 4 - d has
w = d exactly.  Pixel centres sit half a pixel from every edge, far beyond
float32 rounding (about 1e-4 pixel here), so each point's pixel is known
without evaluating the projection under test.
"""
from __future__ import annotations

import math

import numpy as np

from paper_2104_07526_gb300 import scenes

W, H = 640, 480
EYE_Z = 4.0


def camera():
    return scenes.camera((0, 0, EYE_Z), (0, 0, 0), (0, 1, 0), W, H, 60.0)


def point_on_pixel(px: int, py: int, d: float, width=W, height=H, fovy=60.0):
    """World point whose projection is the centre of pixel (px, py) at depth d."""
    t = math.tan(math.radians(fovy) / 2.0)
    aspect = width / height
    ndc_x = 2.0 * (px + 0.5) / width - 1.0
    ndc_y = 2.0 * (py + 0.5) / height - 1.0
    return ndc_x * d * aspect * t, ndc_y * d * t, EYE_Z - d


def pack(xyz: np.ndarray, rgba: np.ndarray) -> np.ndarray:
    """(n,3) coordinates + (n,) rgba words -> (n,4) int32 records."""
    n = xyz.shape[0]
    out = np.empty((n, 4), dtype=np.int32)
    out[:, :3] = xyz.astype(np.float32).view(np.int32)
    out[:, 3] = rgba.astype(np.uint32).view(np.int32)
    return out


def rgba_word(r, g, b, a=255):
    return (np.asarray(r, np.uint32) | (np.asarray(g, np.uint32) << 8) | (np.asarray(b, np.uint32) << 16)
            | (np.uint32(a) << 24)).astype(np.uint32)


def depth_scene(rng: np.random.Generator, npix: int = 400, max_per_pixel: int = 6):
    """Random pixels, each with several points at dyadic depths (multiples of
    1/4 in [1, 6)), some sharing a depth.  Returns (cloud, expected keys) for
    the basic render: per pixel the smallest depth, ties to the smallest
    index, as Sec. 3.1's atomicMin on (depth << 32 | payload) selects."""
    pix = rng.choice(W * H, size=npix, replace=False)
    recs = []
    for p in pix:
        px, py = int(p % W), int(p // W)
        k = int(rng.integers(1, max_per_pixel + 1))
        depths = rng.integers(4, 24, size=k) / 4.0
        if k > 1 and rng.random() < 0.3:
            depths[-1] = depths[0]  # a depth tie
        for d in depths:
            recs.append((p, px, py, float(d)))
    order = rng.permutation(len(recs))
    recs = [recs[i] for i in order]
    xyz = np.array([point_on_pixel(px, py, d) for (_, px, py, d) in recs])
    colour = rng.integers(0, 256, size=(len(recs), 3))
    cloud = pack(xyz, rgba_word(colour[:, 0], colour[:, 1], colour[:, 2]))
    expected = np.full(W * H, np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)
    for i, (p, _, _, d) in enumerate(recs):
        key = (int(np.float32(d).view(np.uint32)) << 32) | i
        if key < int(expected[p]):
            expected[p] = key
    return cloud, expected, recs, colour


def hq_scene(rng: np.random.Generator, npix: int = 300):
    """Per pixel a front depth d0 and further points either inside the 1% band
    (d0 * 257/256, or d0 itself) or clearly outside it (d0 * 33/32).  All
    depths are exact in float32.  Returns (cloud, expected depth bits,
    expected channel sums r, g, b, count)."""
    pix = rng.choice(W * H, size=npix, replace=False)
    recs = []
    for p in pix:
        px, py = int(p % W), int(p // W)
        d0 = float(rng.integers(4, 24)) / 4.0
        recs.append((p, px, py, d0, True))
        for _ in range(int(rng.integers(0, 5))):
            kind = int(rng.integers(0, 3))
            if kind == 0:
                recs.append((p, px, py, d0, True))
            elif kind == 1:
                recs.append((p, px, py, d0 * 257.0 / 256.0, True))
            else:
                recs.append((p, px, py, d0 * 33.0 / 32.0, False))
    order = rng.permutation(len(recs))
    recs = [recs[i] for i in order]
    xyz = np.array([point_on_pixel(px, py, d) for (_, px, py, d, _) in recs])
    colour = rng.integers(0, 256, size=(len(recs), 3))
    cloud = pack(xyz, rgba_word(colour[:, 0], colour[:, 1], colour[:, 2]))
    depth = np.full(W * H, np.uint32(0x7F800000), dtype=np.uint32)
    sums = np.zeros((4, W * H), dtype=np.uint64)
    for (p, _, _, d, _) in recs:
        depth[p] = min(int(depth[p]), int(np.float32(d).view(np.uint32)))
    for i, (p, _, _, d, inside) in enumerate(recs):
        if inside:
            sums[0, p] += colour[i, 0]
            sums[1, p] += colour[i, 1]
            sums[2, p] += colour[i, 2]
            sums[3, p] += 1
    return cloud, depth, sums
