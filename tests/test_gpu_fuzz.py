"""Seeded random cases against the oracle, bit for bit: random clouds (scales
from 1e-4 to 1e5, with NaN, infinite, signed-zero, subnormal and huge
coordinates mixed in), random cameras (perspective, constant-w and
arbitrary 4x4 matrices of random scale, so w ranges over many binades, takes
both signs and lands outside the projection's fast reciprocal window) and
random viewports.  Every exact basic variant, the colour-payload keys, the
HQ buffers (two depth factors), HQS1R's channel sums and the resolves are
compared with the oracle's; so are all five vertex orders of random clouds."""
import numpy as np
import pytest
import torch

import constructed as cs
from gpu_helpers import Renderer, reorder_gpu
from paper_2104_07526_gb300 import pcr, scenes

pytestmark = pytest.mark.gpu

SPECIAL = np.array([np.nan, np.inf, -np.inf, 0.0, -0.0, 1e-40, -1e-40, 3e38, -3e38, 1e-30], dtype=np.float64)


@pytest.fixture(scope="module")
def r():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    rend = Renderer()
    yield rend
    rend.close()


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


@pytest.mark.parametrize("seed", range(32))
def test_random_clouds_cameras_viewports(r, oracle, seed):
    rng = np.random.default_rng(1000 + seed)
    cloud = random_cloud(rng)
    W = int(rng.integers(1, 300))
    H = int(rng.integers(1, 300))
    m = random_matrix(rng, cloud, W, H)
    r.upload(cloud)
    r.view(m, W, H)
    expect = oracle.render_basic(cloud, m, W, H)
    for v in pcr.EXACT_VARIANTS:
        assert np.array_equal(r.render_basic(v), expect), (seed, pcr.VARIANT_NAMES[v])
    bg = int(rng.integers(0, 2 ** 32))
    assert np.array_equal(r.resolve(pcr.PCR_RESOLVE_BASIC, bg), oracle.resolve_basic(expect, cloud, bg)), seed
    rgb = oracle.render_rgb(cloud, m, W, H)
    for v in (pcr.PCR_VARIANT_ATOMICMIN, pcr.PCR_VARIANT_DEDUP_EARLYZ):
        assert np.array_equal(r.render_rgb(v), rgb), (seed, v)
    assert np.array_equal(r.resolve(pcr.PCR_RESOLVE_RGB, bg), oracle.resolve_rgb(rgb, bg)), seed
    for factor in (1.01, float(np.float32(rng.uniform(1.0, 1.5)))):
        e = oracle.render_hq(cloud, m, W, H, factor)
        for v in (pcr.PCR_VARIANT_ATOMICMIN, pcr.PCR_VARIANT_DEDUP_EARLYZ):
            got = r.render_hq(v, factor)
            for a, b in zip(got, e):
                assert np.array_equal(a, b), (seed, factor, v)
        assert np.array_equal(r.resolve(pcr.PCR_RESOLVE_HQ, bg), oracle.resolve_hq(e[1], e[2], bg)), seed
        sums = oracle.hq_channel_sums(cloud, m, W, H, e[0], factor)
        d, *parts = r.render_hq1r_sums(pcr.PCR_VARIANT_DEDUP_EARLYZ, factor)
        assert np.array_equal(d, e[0]), seed
        for a, b in zip(parts, sums):
            assert np.array_equal(a, b), (seed, factor)


@pytest.mark.parametrize("seed", range(16))
def test_random_reorders(r, oracle, seed):
    """Every vertex order on random clouds of random size (tails of both tile
    sizes, 5120 and 6144 keys, and of the 128-point batches), special
    coordinates and degenerate extents included: permutation and records
    against the oracle."""
    rng = np.random.default_rng(2000 + seed)
    cloud = random_cloud(rng)
    if seed % 4 == 3:  # every bulk point on one spot: a zero extent
        bulk = (np.abs(cloud[:, :3].view(np.float32)) < 1e29).all(axis=1)
        cloud[bulk, :3] = cloud[np.argmax(bulk), :3]
    order_seed = int(rng.integers(0, 2 ** 63))
    for mode in (pcr.PCR_ORDER_MORTON, pcr.PCR_ORDER_MORTON_SHUFFLE128, pcr.PCR_ORDER_SHUFFLE,
                 pcr.PCR_ORDER_MORTON63, pcr.PCR_ORDER_MORTON63_SHUFFLE128):
        expect = oracle.reorder(cloud, order_seed, mode)
        dev = torch.from_numpy(cloud.copy()).cuda()
        assert np.array_equal(reorder_gpu(r.h, dev, order_seed, mode), expect), (seed, mode)
        assert np.array_equal(dev.cpu().numpy(), oracle.gather(cloud, expect)), (seed, mode)
