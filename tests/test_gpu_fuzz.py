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

from gpu_helpers import Renderer, reorder_gpu
from paper_2104_07526_gb300 import pcr
from random_inputs import random_cloud, random_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def r():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    rend = Renderer()
    yield rend
    rend.close()


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
