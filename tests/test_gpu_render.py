"""GPU parity: the CUDA render path against the CPU oracle, bit for bit.

Every comparison goes through the C ABI (libpcr.so).  Key buffers, HQ depth
and sum buffers and resolved images are integers, so the bar is exact
equality.
"""
import numpy as np
import pytest
import torch

import constructed as cs
from gpu_helpers import Renderer, U64_EMPTY
from paper_2104_07526_gb300 import pcr, scenes

pytestmark = pytest.mark.gpu

EXACT = pcr.EXACT_VARIANTS
BG = 0x20304050


@pytest.fixture(scope="module")
def r():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    rend = Renderer()
    yield rend
    rend.close()


@pytest.fixture(scope="module")
def sphere():
    # 1M-point recipe at a size the oracle renders in well under a second;
    # 200003 points = 1563 chunks of 128 plus a ragged tail of 35.
    return scenes.sphere_plane(200_003, seed=0).numpy()


def test_sphere1M_config_in_every_order(r, oracle):
    """The 1M-point sphere-and-plane scene at 640x480, as its configuration
    states it, in its generation order and after each one-time reorder: every
    exact variant's keys and the resolved image equal the oracle's."""
    from gpu_helpers import reorder_gpu
    cloud = scenes.sphere_plane(1_000_000, seed=0)
    view = scenes.sphere_plane_views()[0]
    assert (view.width, view.height) == (640, 480)
    dev = cloud.cuda()
    for mode in (None, pcr.PCR_ORDER_MORTON, pcr.PCR_ORDER_MORTON_SHUFFLE128, pcr.PCR_ORDER_SHUFFLE):
        pts = dev.clone()
        if mode is not None:
            reorder_gpu(r.h, pts, 0x5EED, mode)
        host = pts.cpu().numpy()
        expect = oracle.render_basic(host, view.matrix, view.width, view.height)
        img = oracle.resolve_basic(expect, host, 0)
        r.upload(pts)
        r.view(view.matrix, view.width, view.height)
        for v in EXACT:
            assert np.array_equal(r.render_basic(v), expect), (mode, pcr.VARIANT_NAMES[v])
            assert np.array_equal(r.resolve(pcr.PCR_RESOLVE_BASIC, 0), img), (mode, pcr.VARIANT_NAMES[v])


def test_sphere_plane_all_variants(r, oracle, sphere):
    view = scenes.sphere_plane_views()[0]
    expect = oracle.render_basic(sphere, view.matrix, view.width, view.height)
    img_expect = oracle.resolve_basic(expect, sphere, 0x12345678)
    r.upload(sphere)
    r.view(view.matrix, view.width, view.height)
    assert (expect != U64_EMPTY).sum() > 10000
    for v in EXACT:
        got = r.render_basic(v)
        assert np.array_equal(got, expect), pcr.VARIANT_NAMES[v]
        img = r.resolve(pcr.PCR_RESOLVE_BASIC, 0x12345678)
        assert np.array_equal(img, img_expect), pcr.VARIANT_NAMES[v]


def test_constructed_depth_scene(r):
    rng = np.random.default_rng(21)
    cloud, expected, _, _ = cs.depth_scene(rng, npix=3000, max_per_pixel=8)
    r.upload(cloud)
    r.view(cs.camera(), cs.W, cs.H)
    for v in EXACT:
        assert np.array_equal(r.render_basic(v), expected), pcr.VARIANT_NAMES[v]


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, 127, 128, 129, 4097])
def test_ragged_sizes(r, oracle, n):
    cloud = scenes.random_cloud(n, seed=n + 100).numpy() if n else np.zeros((0, 4), np.int32)
    m = scenes.camera((0.2, -2.6, 1.4), (0, 0, 0), (0, 0, 1), 32, 24)
    expect = oracle.render_basic(cloud, m, 32, 24)
    r.upload(cloud)
    r.view(m, 32, 24)
    for v in EXACT:
        assert np.array_equal(r.render_basic(v), expect), (n, pcr.VARIANT_NAMES[v])


def test_single_pixel_contention(r, oracle):
    """All points on one pixel: distinct depths, then equal depths (the
    smallest index must win), across many warps and blocks."""
    n = 300_000
    rng = np.random.default_rng(5)
    d = rng.integers(4, 4000, size=n) / 256.0  # exact dyadic depths
    xyz = np.stack([np.zeros(n), np.zeros(n), cs.EYE_Z - d], 1)
    cloud = cs.pack(xyz, np.arange(n, dtype=np.uint32))
    r.upload(cloud)
    r.view(cs.camera(), cs.W, cs.H)
    expect = oracle.render_basic(cloud, cs.camera(), cs.W, cs.H)
    for v in EXACT:
        assert np.array_equal(r.render_basic(v), expect), pcr.VARIANT_NAMES[v]
    same = cs.pack(np.tile([[0.0, 0.0, 1.5]], (n, 1)), np.arange(n, dtype=np.uint32))
    r.upload(same)
    for v in EXACT:
        got = r.render_basic(v)
        assert got[cs.W // 2 + (cs.H // 2) * cs.W] == (int(np.float32(2.5).view(np.uint32)) << 32), v


def test_culling_edge_inputs(r, oracle):
    """NaN and infinite coordinates, points behind the eye, points exactly
    on the viewport edges."""
    t = np.tan(np.radians(30.0))
    rows = [[np.nan, 0, 0], [0, np.inf, 0], [0, 0, -np.inf], [0, 0, 9.0], [0, 0, 4.0],
            [t * 2.0 * 4 / 3, 0, 2.0], [-t * 2.0 * 4 / 3, 0, 2.0], [0, t * 2.0, 2.0], [0, -t * 2.0, 2.0],
            [1e30, 1e30, -1e30], [1e-30, -1e-30, 3.9999], [0.1, 0.1, 3.0]]
    cloud = cs.pack(np.array(rows, dtype=np.float64), np.arange(len(rows), dtype=np.uint32))
    r.upload(cloud)
    r.view(cs.camera(), cs.W, cs.H)
    expect = oracle.render_basic(cloud, cs.camera(), cs.W, cs.H)
    for v in EXACT:
        assert np.array_equal(r.render_basic(v), expect), pcr.VARIANT_NAMES[v]


def test_tiny_and_wide_viewports(r, oracle):
    cloud = scenes.random_cloud(50_000, seed=3).numpy()
    for (W, H) in [(1, 1), (3, 1), (1, 5), (16384, 2), (2, 16384)]:
        m = scenes.camera((0.1, -3.0, 0.2), (0, 0, 0), (0, 0, 1), W, H, 75.0)
        expect = oracle.render_basic(cloud, m, W, H)
        r.upload(cloud)
        r.view(m, W, H)
        for v in (pcr.PCR_VARIANT_ATOMICMIN, pcr.PCR_VARIANT_DEDUP_EARLYZ, pcr.PCR_VARIANT_REDUCE_EARLYZ):
            assert np.array_equal(r.render_basic(v), expect), (W, H, v)


def test_largest_viewport(r, oracle):
    """The largest viewport the interface takes, 16384 x 16384 (2^28 pixels:
    pixel indices near the top of their 32-bit range, a 2 GB key buffer),
    bit-exact for the basic variants, the HQ buffers and the resolve."""
    W = H = 16384
    cloud = scenes.sphere_plane(200_003, seed=21).numpy()
    m = scenes.camera((0, 0, 4), (0, 0, 0), (0, 1, 0), W, H, 90.0)
    r.upload(cloud)
    r.view(m, W, H)
    expect = oracle.render_basic(cloud, m, W, H)
    covered = np.nonzero(expect != U64_EMPTY)[0]
    assert covered.size > 100_000 and covered.max() > (1 << 27)  # pixels in the upper half of the range
    for v in (pcr.PCR_VARIANT_ATOMICMIN, pcr.PCR_VARIANT_EARLYZ, pcr.PCR_VARIANT_DEDUP_EARLYZ):
        assert np.array_equal(r.render_basic(v), expect), v
    pcr.pcr_resolve(r.h, pcr.PCR_RESOLVE_BASIC, r.fb["image"], 0x11223344)
    torch.cuda.synchronize()
    assert np.array_equal(r.fb["image"].cpu().numpy().view(np.uint32),
                          oracle.resolve_basic(expect, cloud, 0x11223344))
    del expect
    got = r.render_hq(pcr.PCR_VARIANT_DEDUP_EARLYZ)
    for a, b in zip(got, oracle.render_hq(cloud, m, W, H, 1.01)):
        assert np.array_equal(a, b)


def test_no_clear_accumulates(r, oracle, sphere):
    """clear=0 merges by minimum: rendering the same cloud twice equals once,
    and a buffer pre-filled with keys keeps the smaller of old and new."""
    view = scenes.sphere_plane_views()[0]
    r.upload(sphere)
    r.view(view.matrix, view.width, view.height)
    once = r.render_basic(pcr.PCR_VARIANT_DEDUP_EARLYZ)
    twice = r.render_basic(pcr.PCR_VARIANT_EARLYZ, clear=False)
    assert np.array_equal(once, twice)
    prefill = np.full(once.size, np.uint64((int(np.float32(4.0).view(np.uint32)) << 32) | 7), np.uint64)
    r.fb["keys"].copy_(torch.from_numpy(prefill.view(np.int64)))
    got = r.render_basic(pcr.PCR_VARIANT_DEDUP, clear=False)
    assert np.array_equal(got, np.minimum(prefill, once))


def test_just_set_writes_valid_keys(r, oracle, sphere):
    """Sec. 5 just-set has no depth test: each covered pixel holds the key of
    some point that lands there, and the covered set equals the oracle's."""
    view = scenes.sphere_plane_views()[0]
    expect = oracle.render_basic(sphere, view.matrix, view.width, view.height)
    r.upload(sphere)
    r.view(view.matrix, view.width, view.height)
    got = r.render_basic(pcr.PCR_VARIANT_JUST_SET)
    assert np.array_equal(got == U64_EMPTY, expect == U64_EMPTY)
    hit = np.nonzero(got != U64_EMPTY)[0]
    idx = (got[hit] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    p = np.ascontiguousarray(sphere[:, :3]).view(np.float32)
    for j in range(0, hit.size, max(1, hit.size // 2000)):
        pr = oracle.project(view.matrix, view.width, view.height, *p[idx[j]])
        assert pr is not None and pr[0] == hit[j]
        assert int(got[hit[j]]) >> 32 == int(np.float32(pr[1]).view(np.uint32))


def test_resolve_out_of_range_index(r):
    """A key naming a point outside the cloud resolves to the background and
    raises bit 0 of the device error word."""
    cloud = cs.pack(np.zeros((4, 3)), np.array([1, 2, 3, 4], dtype=np.uint32))
    r.upload(cloud)
    r.view(np.eye(4, dtype=np.float32), 2, 2)
    assert pcr.pcr_last_device_error(r.h) == 0
    keys = np.array([0xFFFFFFFFFFFFFFFF, (0x3F800000 << 32) | 2, (0x3F800000 << 32) | 4, 5], dtype=np.uint64)
    r.fb["keys"].copy_(torch.from_numpy(keys.view(np.int64)))
    img = r.resolve(pcr.PCR_RESOLVE_BASIC, 0xDEADBEEF)
    assert img.tolist() == [0xDEADBEEF, 3, 0xDEADBEEF, 0xDEADBEEF]
    assert pcr.pcr_last_device_error(r.h) == 1
    assert pcr.pcr_last_device_error(r.h) == 0


# --- Sec. 3.5 ------------------------------------------------------------------

def test_hq_constructed(r):
    rng = np.random.default_rng(8)
    cloud, depth, sums = cs.hq_scene(rng, npix=4000)
    r.upload(cloud)
    r.view(cs.camera(), cs.W, cs.H)
    for v in (0, 1, 2, 3):
        d, rg, ba = r.render_hq(v, 1.01)
        assert np.array_equal(d, depth), v
        assert np.array_equal(rg, (sums[0] << np.uint64(32)) | sums[1]), v
        assert np.array_equal(ba, (sums[2] << np.uint64(32)) | sums[3]), v


def test_hq_sphere_parity(r, oracle, sphere):
    view = scenes.sphere_plane_views()[0]
    W, H = view.width, view.height
    r.upload(sphere)
    r.view(view.matrix, W, H)
    for factor in (1.01, 1.0, 1.5):
        e = oracle.render_hq(sphere, view.matrix, W, H, factor)
        img0 = oracle.resolve_hq(e[1], e[2], 0x01020304)
        for v in (0, 1, 2, 3):
            got = r.render_hq(v, factor)
            for a, b in zip(got, e):
                assert np.array_equal(a, b), (v, factor)
            img = r.resolve(pcr.PCR_RESOLVE_HQ, 0x01020304)
            assert np.array_equal(img, img0), (v, factor)


def test_hq_single_pixel_heavy(r, oracle):
    """200k points on one pixel within the band: 32-bit sums stay exact and
    the warp aggregation adds up exactly."""
    n = 200_000
    rng = np.random.default_rng(9)
    d = 2.0 + rng.integers(0, 4, size=n) / 1024.0
    xyz = np.stack([np.zeros(n), np.zeros(n), cs.EYE_Z - d], 1)
    col = rng.integers(0, 256, size=(n, 3))
    cloud = cs.pack(xyz, cs.rgba_word(col[:, 0], col[:, 1], col[:, 2]))
    r.upload(cloud)
    r.view(cs.camera(), cs.W, cs.H)
    e = oracle.render_hq(cloud, cs.camera(), cs.W, cs.H, 1.01)
    for v in (0, 3):
        got = r.render_hq(v, 1.01)
        for a, b in zip(got, e):
            assert np.array_equal(a, b), v
    p = cs.W // 2 + (cs.H // 2) * cs.W
    assert int(e[2][p]) & 0xFFFFFFFF == n


def test_hq_ragged(r, oracle):
    for n in (0, 1, 33, 129, 5000):
        cloud = scenes.random_cloud(n, seed=n).numpy() if n else np.zeros((0, 4), np.int32)
        m = scenes.camera((0.3, -2.2, 1.0), (0, 0, 0), (0, 0, 1), 20, 15)
        e = oracle.render_hq(cloud, m, 20, 15, 1.01)
        r.upload(cloud)
        r.view(m, 20, 15)
        for v in (0, 3):
            got = r.render_hq(v, 1.01)
            for a, b in zip(got, e):
                assert np.array_equal(a, b), (n, v)


# --- Sec. 3.5.1 HQS1R -----------------------------------------------------------

def _hq1r_check(r, oracle, cloud, m, W, H, factor=1.01, variants=(0, 1, 2, 3)):
    d0, rg0, ba0 = oracle.render_hq(cloud, m, W, H, factor)
    sums = oracle.hq_channel_sums(cloud, m, W, H, d0, factor)
    img0 = oracle.resolve_hq(rg0, ba0, 0x0A0B0C0D)
    for v in variants:
        d, *got = r.render_hq1r_sums(v, factor)
        assert np.array_equal(d, d0), v
        for a, b in zip(got, sums):
            assert np.array_equal(a, b), v
        assert np.array_equal(r.resolve(pcr.PCR_RESOLVE_HQ1R, 0x0A0B0C0D), img0), v


def test_hq1r_sphere(r, oracle, sphere):
    view = scenes.sphere_plane_views()[0]
    r.upload(sphere)
    r.view(view.matrix, view.width, view.height)
    _hq1r_check(r, oracle, sphere, view.matrix, view.width, view.height)


def test_hq1r_constructed_and_ragged(r, oracle):
    rng = np.random.default_rng(12)
    cloud, _, _ = cs.hq_scene(rng, npix=3000)
    r.upload(cloud)
    r.view(cs.camera(), cs.W, cs.H)
    _hq1r_check(r, oracle, cloud, cs.camera(), cs.W, cs.H)
    for n in (0, 1, 129):
        small = scenes.random_cloud(n, seed=n).numpy() if n else np.zeros((0, 4), np.int32)
        m = scenes.camera((0.3, -2.2, 1.0), (0, 0, 0), (0, 0, 1), 20, 15)
        r.upload(small)
        r.view(m, 20, 15)
        _hq1r_check(r, oracle, small, m, 20, 15, variants=(0, 3))


def test_hq1r_overflow_protocol(r, oracle):
    """Hundreds of thousands of points on a few pixels: the primary word
    crosses its 64-point limit again and again; every contribution must still
    be counted exactly once."""
    n = 400_000
    rng = np.random.default_rng(13)
    px = rng.integers(0, 3, size=n)
    d = 2.0 + rng.integers(0, 4, size=n) / 1024.0
    pts = np.stack([cs.point_on_pixel(300 + int(k), 200, 2.0) for k in range(3)])
    xyz = pts[px].copy()
    xyz[:, 2] = cs.EYE_Z - d
    # keep the pixel: scale x, y with the depth so each point stays on its ray
    xyz[:, 0] *= d / 2.0
    xyz[:, 1] *= d / 2.0
    col = rng.integers(0, 256, size=(n, 3))
    cloud = cs.pack(xyz, cs.rgba_word(col[:, 0], col[:, 1], col[:, 2]))
    r.upload(cloud)
    r.view(cs.camera(), cs.W, cs.H)
    _hq1r_check(r, oracle, cloud, cs.camera(), cs.W, cs.H)
    d0, *_ = oracle.render_hq(cloud, cs.camera(), cs.W, cs.H, 1.01)
    counts = oracle.hq_channel_sums(cloud, cs.camera(), cs.W, cs.H, d0, 1.01)[3]
    assert sorted(counts[counts > 0].tolist())[-1] > 100_000  # heavy pixels really were exercised


def test_hq1r_groups_larger_than_a_word(r, oracle):
    """Points sorted by pixel, in runs of every length from 1 to 300: warp
    groups of up to 128 points (more than the 64 a primary word holds, which
    go to the fallback sums directly) next to small ones that use the word."""
    rng = np.random.default_rng(14)
    runs = np.concatenate([np.arange(1, 301), rng.integers(1, 400, size=700)])
    px = np.repeat(np.arange(runs.size) % 5, runs)
    n = px.size
    d = 2.0 + rng.integers(0, 4, size=n) / 1024.0
    pts = np.stack([cs.point_on_pixel(100 + 7 * int(k), 60 + 3 * int(k), 2.0) for k in range(5)])
    xyz = pts[px].copy()
    xyz[:, 2] = cs.EYE_Z - d
    xyz[:, 0] *= d / 2.0
    xyz[:, 1] *= d / 2.0
    col = rng.integers(0, 256, size=(n, 3))
    cloud = cs.pack(xyz, cs.rgba_word(col[:, 0], col[:, 1], col[:, 2]))
    r.upload(cloud)
    r.view(cs.camera(), cs.W, cs.H)
    _hq1r_check(r, oracle, cloud, cs.camera(), cs.W, cs.H)
    # the same sums through the two-atomic HQ pass
    d0, rg0, ba0 = oracle.render_hq(cloud, cs.camera(), cs.W, cs.H, 1.01)
    for v in (0, 1, 2, 3):
        got = r.render_hq(v, 1.01)
        for a, b in zip(got, (d0, rg0, ba0)):
            assert np.array_equal(a, b), v


def test_host_upload_and_download(r, oracle, sphere):
    """The e2e path: points copied from pinned host memory by the library,
    the frame rendered, the image read back into host memory."""
    view = scenes.sphere_plane_views()[0]
    W, H = view.width, view.height
    host = torch.from_numpy(np.ascontiguousarray(sphere)).pin_memory()
    dev = torch.zeros_like(host, device="cuda")
    r.view(view.matrix, W, H)
    pcr.pcr_upload_points_from_host(r.h, dev, host, host.shape[0])
    r.points, r.n = dev, host.shape[0]
    pcr.pcr_clear(r.h, pcr.PCR_CLEAR_KEYS)
    pcr.pcr_render_basic(r.h, pcr.PCR_VARIANT_EARLYZ, False)
    pcr.pcr_resolve(r.h, pcr.PCR_RESOLVE_BASIC, r.fb["image"], 0x0F0F0F0F)
    img = np.empty(W * H, dtype=np.uint32)
    pcr.pcr_download(r.h, img, r.fb["image"])
    expect = oracle.render_basic(sphere, view.matrix, W, H)
    assert np.array_equal(img, oracle.resolve_basic(expect, sphere, 0x0F0F0F0F))
    assert torch.equal(dev.cpu(), host)


def test_render_from_mapped_host_memory(r, oracle, sphere):
    """Points left in pinned host memory and read by the render kernels over
    the host link: every exact variant and the resolve's colour gather match
    the oracle."""
    view = scenes.sphere_plane_views()[0]
    W, H = view.width, view.height
    host = torch.from_numpy(np.ascontiguousarray(sphere)).pin_memory()
    n = host.shape[0]
    r.view(view.matrix, W, H)
    pcr.pcr_upload_points_mapped(r.h, host, n)
    expect = oracle.render_basic(sphere, view.matrix, W, H)
    for v in pcr.EXACT_VARIANTS:
        pcr.pcr_render_basic(r.h, v, True)
        assert np.array_equal(r.fb["keys"].cpu().numpy().view(np.uint64), expect), pcr.VARIANT_NAMES[v]
    pcr.pcr_resolve(r.h, pcr.PCR_RESOLVE_BASIC, r.fb["image"], 0)
    assert np.array_equal(r.fb["image"].cpu().numpy().view(np.uint32), oracle.resolve_basic(expect, sphere, 0))
    torch.cuda.synchronize()
    pcr.pcr_upload_points_mapped(r.h, host[:0], 0)  # n = 0 is allowed


def test_mapped_upload_refusals(r):
    """Pageable host memory, device memory, a misaligned start and a range
    running past the pinned block are refused before anything is launched."""
    host = torch.zeros((1024, 4), dtype=torch.int32).pin_memory()
    pageable = torch.zeros((1024, 4), dtype=torch.int32)
    dev = torch.zeros((1024, 4), dtype=torch.int32, device="cuda")
    lib = pcr.lib()
    assert lib.pcr_upload_points_mapped(r.h, pageable.data_ptr(), 1024) == pcr.PCR_ERR_ARG
    assert lib.pcr_upload_points_mapped(r.h, dev.data_ptr(), 1024) == pcr.PCR_ERR_ARG
    assert lib.pcr_upload_points_mapped(r.h, host.data_ptr() + 4, 1000) == pcr.PCR_ERR_ARG
    assert lib.pcr_upload_points_mapped(r.h, host.data_ptr(), 1 << 31) == pcr.PCR_ERR_ARG
    assert lib.pcr_upload_points_mapped(r.h, None, 1) == pcr.PCR_ERR_ARG
    assert lib.pcr_upload_points_mapped(r.h, host.data_ptr(), 1024) == pcr.PCR_OK
    r.upload(np.zeros((0, 4), np.int32))


def test_captured_frames_replay_exactly(oracle):
    """pcr_capture_begin / _end record a frame (clear + render + resolve, and
    an HQ frame) into a graph; each replay gives the oracle's buffers.  While
    recording, calls that synchronise or copy from the host are refused and
    nothing runs; an unfinished capture is dropped by pcr_destroy."""
    from gpu_helpers import ensure_built
    ensure_built()
    cloud = scenes.sphere_plane(100_003, seed=13).numpy()
    W, H = 320, 240
    m = scenes.camera((0, 0, 4), (0, 0, 0), (0, 1, 0), W, H)
    pts = torch.from_numpy(cloud.copy()).cuda()
    fb = pcr.alloc_framebuffer(W, H)
    hq_image = torch.empty(W * H, dtype=torch.int32, device="cuda")
    expect = oracle.render_basic(cloud, m, W, H)
    _, rg, ba = oracle.render_hq(cloud, m, W, H, 1.01)
    with pcr.Context(0, stream=torch.cuda.current_stream()) as c:
        h = c.handle
        pcr.pcr_upload_points(h, pts, pts.shape[0])
        pcr.pcr_set_matrix(h, m)
        pcr.pcr_set_viewport(h, W, H)
        pcr.pcr_set_framebuffer(h, fb["keys"], fb["hq_depth"], fb["hq_rg"], fb["hq_ba"])
        with pytest.raises(pcr.PcrError):
            pcr.pcr_capture_end(h)  # nothing open
        pcr.pcr_capture_begin(h)
        with pytest.raises(pcr.PcrError):
            pcr.pcr_capture_begin(h)  # already open
        for refused in (lambda: pcr.pcr_synchronize(h), lambda: pcr.pcr_last_device_error(h),
                        lambda: pcr.pcr_set_stream(h, torch.cuda.current_stream())):
            with pytest.raises(pcr.PcrError) as e:
                refused()
            assert e.value.status == pcr.PCR_ERR_ARG
        pcr.pcr_clear(h, pcr.PCR_CLEAR_KEYS)
        pcr.pcr_render_basic(h, pcr.PCR_VARIANT_DEDUP_EARLYZ, False)
        pcr.pcr_resolve(h, pcr.PCR_RESOLVE_BASIC, fb["image"], BG)
        pcr.pcr_render_hq(h, 1.01, pcr.PCR_VARIANT_DEDUP_EARLYZ, True)
        pcr.pcr_resolve(h, pcr.PCR_RESOLVE_HQ, hq_image, BG)
        g = pcr.pcr_capture_end(h)
        try:
            for rep in range(3):
                for t in (fb["keys"], fb["image"], fb["hq_rg"], hq_image):
                    t.fill_(0x5A5A5A5A)
                pcr.pcr_graph_launch(h, g)
                torch.cuda.synchronize()
                assert np.array_equal(fb["keys"].cpu().numpy().view(np.uint64), expect), rep
                assert np.array_equal(fb["image"].cpu().numpy().view(np.uint32),
                                      oracle.resolve_basic(expect, cloud, BG)), rep
                assert np.array_equal(fb["hq_rg"].cpu().numpy().view(np.uint64), rg), rep
                assert np.array_equal(hq_image.cpu().numpy().view(np.uint32), oracle.resolve_hq(rg, ba, BG)), rep
        finally:
            pcr.pcr_graph_destroy(g)
        assert pcr.pcr_last_device_error(h) == 0  # the context is usable again after the capture
    with pcr.Context(0, stream=torch.cuda.current_stream()) as c2:
        pcr.pcr_capture_begin(c2.handle)  # left open: pcr_destroy drops it
