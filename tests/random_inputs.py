"""Seeded random test inputs: point clouds with special coordinates mixed in,
and cameras or arbitrary 4x4 matrices aimed at a cloud's bulk.  Inputs
only: nothing here computes any part of the rendering method."""
import numpy as np

import constructed as cs
from paper_2104_07526_gb300 import scenes

SPECIAL = np.array([np.nan, np.inf, -np.inf, 0.0, -0.0, 1e-40, -1e-40, 3e38, -3e38, 1e-30], dtype=np.float64)


def random_cloud(rng: np.random.Generator) -> np.ndarray:
    n = int(rng.integers(1, 30_000))
    scale = 10.0 ** rng.uniform(-4.0, 5.0)
    xyz = rng.uniform(-scale, scale, size=(n, 3)) + rng.uniform(-scale, scale, size=3)
    # a few points on a shared plane and a few duplicates: equal depths
    k = n // 20
    if k:
        xyz[rng.integers(0, n, k), 2] = xyz[0, 2]
        xyz[rng.integers(0, n, k)] = xyz[rng.integers(0, n, k)]
    # special coordinates in about 2% of the points
    s = n // 50
    if s:
        xyz[rng.integers(0, n, s), rng.integers(0, 3, s)] = rng.choice(SPECIAL, s)
    rgba = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    return cs.pack(xyz, rgba)


def random_matrix(rng: np.random.Generator, cloud: np.ndarray, width: int, height: int) -> np.ndarray:
    kind = int(rng.integers(0, 3))
    # aimed at the bulk of the cloud: a centre and spread that ignore the
    # special coordinates
    xyz = cloud[:, :3].view(np.float32).astype(np.float64)
    bulk = xyz[(np.abs(xyz) < 1e29).all(axis=1)]
    centre = np.median(bulk, axis=0) if len(bulk) else np.zeros(3)
    extent = float(np.percentile(np.abs(bulk - centre).max(axis=1), 90)) if len(bulk) else 1.0
    extent = extent if extent > 0 else 1.0
    if kind == 0:  # a perspective camera somewhere around the cloud
        eye = centre + rng.normal(size=3) * extent * rng.uniform(0.2, 4.0)
        target = centre + rng.normal(size=3) * extent * 0.3
        up = rng.normal(size=3)
        return scenes.camera(tuple(eye), tuple(target), tuple(up), width, height, float(rng.uniform(5.0, 160.0)))
    m = rng.normal(size=(4, 4)) / extent
    if kind == 1:  # constant w: many equal depths, ties go by index
        m[3] = [0.0, 0.0, 0.0, rng.uniform(0.5, 2.0)]
    # scales down to 1e-14: w below 2^-40 as well as above 2^40
    m *= 10.0 ** rng.uniform(-14.0, 6.0)
    return m.astype(np.float32)
