"""Full-size GPU parity: the 50M-point boxes scene on all variants and
cameras, and the 800M-point scan scene in the launch configuration the
benchmark times (shuffled-Morton order, overview camera, 1920x1080,
early-z), compared with the oracle over whole buffers, with every exact
variant, the busy-loop, the colour payload and the HQ passes."""
import numpy as np
import pytest
import torch

from gpu_helpers import Renderer
from paper_2104_07526_gb300 import pcr, scenes

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

BENCH_SEED = 0x5EED  # the reorder seed bench.py uses


@pytest.fixture(scope="module")
def r():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    rend = Renderer()
    yield rend
    rend.close()


def test_boxes50M_all_variants_all_cameras(r, oracle):
    cloud = scenes.boxes(50_000_000, seed=0).numpy()
    r.upload(cloud)
    for view in scenes.boxes_views(0):
        W, H = view.width, view.height
        r.view(view.matrix, W, H)
        expect = oracle.render_basic(cloud, view.matrix, W, H)
        assert (expect != np.uint64(2 ** 64 - 1)).sum() > 100_000, view.name
        for v in pcr.EXACT_VARIANTS:
            assert np.array_equal(r.render_basic(v), expect), (view.name, pcr.VARIANT_NAMES[v])
        img = r.resolve(pcr.PCR_RESOLVE_BASIC, 0x00FF00FF)
        assert np.array_equal(img, oracle.resolve_basic(expect, cloud, 0x00FF00FF)), view.name
        e = oracle.render_hq(cloud, view.matrix, W, H, 1.01)
        for v in (0, 1, 2, 3):
            got = r.render_hq(v, 1.01)
            for a, b in zip(got, e):
                assert np.array_equal(a, b), (view.name, v)
        img = r.resolve(pcr.PCR_RESOLVE_HQ, 0x00FF00FF)
        assert np.array_equal(img, oracle.resolve_hq(e[1], e[2], 0x00FF00FF)), view.name


def test_scan800M_bench_configuration(r, oracle):
    n = 800_000_000
    original = scenes.scan(n, seed=0, device="cuda")
    views = {v.name: v for v in scenes.scan_views(n, 0)}
    h = r.h
    ws = torch.empty(pcr.pcr_reorder_workspace_size(n), dtype=torch.uint8, device="cuda")

    # Morton order (A11, A12): a stable sort by the oracle's codes.
    morton = original.clone()
    perm_m = torch.empty(n, dtype=torch.int32, device="cuda")
    pcr.pcr_reorder_morton_shuffle128(h, morton, n, BENCH_SEED, pcr.PCR_ORDER_MORTON, ws, perm_m)
    # Shuffled Morton (A13), the benchmark's order.
    cloud = original.clone()
    perm_s = torch.empty(n, dtype=torch.int32, device="cuda")
    pcr.pcr_reorder_morton_shuffle128(h, cloud, n, BENCH_SEED, pcr.PCR_ORDER_MORTON_SHUFFLE128, ws, perm_s)
    torch.cuda.synchronize()
    del ws
    for perm in (perm_m, perm_s):  # each is a permutation of 0..n-1
        seen = torch.zeros(n, dtype=torch.uint8, device="cuda")
        seen[perm.long()] = 1
        assert bool(seen.all())
        del seen
    assert torch.equal(morton, original[perm_m.long()])
    assert torch.equal(cloud, original[perm_s.long()])
    del morton
    host_orig = original.cpu().numpy()
    del original
    torch.cuda.empty_cache()

    pm = perm_m.cpu().numpy().view(np.uint32)
    ps = perm_s.cpu().numpy().view(np.uint32)
    del perm_m, perm_s
    codes = oracle.morton_codes(host_orig)[pm]
    dc = np.diff(codes.astype(np.int64))
    assert (dc >= 0).all()
    assert (np.diff(pm.astype(np.int64))[dc == 0] > 0).all()  # stable: ties keep input order
    del codes, dc
    nb = (n + 127) // 128
    order = np.argsort(oracle.counter_keys(BENCH_SEED, nb), kind="stable")
    idx = (order[:, None].astype(np.int64) * 128 + np.arange(128)[None, :]).reshape(-1)
    expect_s = pm[idx[idx < n]]
    assert np.array_equal(ps, expect_s)
    del idx, expect_s, pm, ps

    # The frame the benchmark times: whole key buffer, image and HQ buffers.
    host = cloud.cpu().numpy()
    del host_orig
    view = views["overview"]
    W, H = view.width, view.height
    pcr.pcr_upload_points(h, cloud, n)
    r.points = cloud
    r.n = n
    r.view(view.matrix, W, H)
    expect = oracle.render_basic(host, view.matrix, W, H)
    got = r.render_basic(pcr.PCR_VARIANT_DEDUP_EARLYZ)
    assert (expect != np.uint64(2 ** 64 - 1)).sum() > 200_000  # about 324k covered pixels
    assert np.array_equal(got, expect)
    assert np.array_equal(r.resolve(pcr.PCR_RESOLVE_BASIC, 0), oracle.resolve_basic(expect, host, 0))
    for v in (pcr.PCR_VARIANT_ATOMICMIN, pcr.PCR_VARIANT_EARLYZ, pcr.PCR_VARIANT_REDUCE_EARLYZ):
        assert np.array_equal(r.render_basic(v), expect), pcr.VARIANT_NAMES[v]
    # the busy-loop comparison kernel and the colour-payload keys, full size
    assert np.array_equal(r.render_basic(pcr.PCR_VARIANT_BUSY_LOOP), expect)
    assert pcr.pcr_last_device_error(h) == 0
    assert np.array_equal(r.render_rgb(pcr.PCR_VARIANT_EARLYZ), oracle.render_rgb(host, view.matrix, W, H))
    e = oracle.render_hq(host, view.matrix, W, H, 1.01)
    got = r.render_hq(pcr.PCR_VARIANT_DEDUP_EARLYZ, 1.01)
    for a, b in zip(got, e):
        assert np.array_equal(a, b)
    # HQS1R: its primary words plus fallback sums give the same channel sums
    sums = oracle.hq_channel_sums(host, view.matrix, W, H, e[0], 1.01)
    d, *parts = r.render_hq1r_sums(pcr.PCR_VARIANT_DEDUP_EARLYZ, 1.01)
    assert np.array_equal(d, e[0])
    for a, b in zip(parts, sums):
        assert np.array_equal(a, b)
    # the other two cameras with the benchmark's variant and dedup+early-z
    for name in ("closeup", "empty"):
        vv = views[name]
        r.view(vv.matrix, vv.width, vv.height)
        want = oracle.render_basic(host, vv.matrix, vv.width, vv.height)
        for v in (pcr.PCR_VARIANT_EARLYZ, pcr.PCR_VARIANT_DEDUP_EARLYZ):
            assert np.array_equal(r.render_basic(v), want), (name, pcr.VARIANT_NAMES[v])
