"""The debug build (libpcr_debug.so, PCR_DEBUG): its kernel counters show
the paper's stated behaviour of the variants, and its device bounds checks
stay silent on correct renders whose buffers equal the release build's.

Sec. 3.4: warp deduplication sends one atomic per distinct pixel per warp
row.  The kernels walk rows of 32 consecutive points (chunks of four rows),
so the expected count follows from the oracle's projection of every point.
A chunk whose first row holds more than 16 runs of pixels skips the match
(its pixels are nearly all distinct); there every visible point writes, and
the expected count says so.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest
import torch

from paper_2104_07526_gb300 import build, pcr, scenes

pytestmark = pytest.mark.gpu

NO_PIXEL = 0xFFFFFFFF
MAX_RUNS = 16


class DebugRenderer:
    """A context of the debug library on torch's current stream."""

    def __init__(self):
        build.build(debug=True)
        self.L = pcr.load_library(pcr.DEBUG_LIB_PATH)
        h = C.c_void_p()
        self._ok(self.L.pcr_create(C.byref(h), 0))
        self.h = h.value
        self._ok(self.L.pcr_set_stream(self.h, torch.cuda.current_stream().cuda_stream))

    @staticmethod
    def _ok(status):
        assert status == pcr.PCR_OK, pcr.pcr_status_string(status)

    def close(self):
        self.L.pcr_destroy(self.h)

    def setup(self, cloud: np.ndarray, m, W: int, H: int):
        self.points = torch.from_numpy(np.ascontiguousarray(cloud)).cuda()
        self.n = cloud.shape[0]
        self._ok(self.L.pcr_upload_points(self.h, self.points.data_ptr(), self.n))
        mm = np.ascontiguousarray(np.asarray(m, dtype=np.float32).reshape(16))
        self._ok(self.L.pcr_set_matrix(self.h, mm.ctypes.data_as(C.POINTER(C.c_float))))
        self._ok(self.L.pcr_set_viewport(self.h, W, H))
        self.fb = pcr.alloc_framebuffer(W, H, "cuda")
        self._ok(self.L.pcr_set_framebuffer(self.h, self.fb["keys"].data_ptr(), self.fb["hq_depth"].data_ptr(),
                                            self.fb["hq_rg"].data_ptr(), self.fb["hq_ba"].data_ptr()))

    def counters(self) -> list[int]:
        out = (C.c_uint64 * 4)()
        self._ok(self.L.pcr_debug_counters(self.h, out))
        return list(out)

    def error_word(self) -> int:
        code = C.c_uint32()
        self._ok(self.L.pcr_last_device_error(self.h, C.byref(code)))
        return code.value

    def render_basic(self, variant: int):
        self.counters()  # clear
        self._ok(self.L.pcr_render_basic(self.h, variant, 1))
        torch.cuda.synchronize()
        return self.fb["keys"].cpu().numpy().view(np.uint64), self.counters()

    def render_hq(self, variant: int):
        self.counters()
        self._ok(self.L.pcr_render_hq(self.h, C.c_float(1.01), variant, 1))
        torch.cuda.synchronize()
        bufs = [self.fb[k].cpu().numpy() for k in ("hq_depth", "hq_rg", "hq_ba")]
        return [bufs[0].view(np.uint32), bufs[1].view(np.uint64), bufs[2].view(np.uint64)], self.counters()


@pytest.fixture(scope="module")
def dbg():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    r = DebugRenderer()
    yield r
    r.close()


def _pixels(oracle, pts: np.ndarray, m, W: int, H: int) -> np.ndarray:
    """Pixel of every point by the oracle's projection, NO_PIXEL if culled."""
    xyz = pts[:, :3].view(np.float32)
    out = np.full(pts.shape[0], NO_PIXEL, dtype=np.int64)
    for i, (x, y, z) in enumerate(xyz.tolist()):
        p = oracle.project(m, W, H, x, y, z)
        if p is not None:
            out[i] = p[0]
    return out


def _expected_dedup_writes(pix: np.ndarray) -> int:
    """One write per distinct visible pixel per row of 32 points; every
    visible point of a chunk (4 rows) whose first row has more than 16 runs."""
    n = pix.size
    chunks = (n + 127) // 128
    padded = np.full(chunks * 128, NO_PIXEL, dtype=np.int64)
    padded[:n] = pix
    total = 0
    for c in range(chunks):
        rows = padded[c * 128:(c + 1) * 128].reshape(4, 32)
        r0 = rows[0]
        vis0 = r0 != NO_PIXEL
        prev = np.concatenate([[NO_PIXEL], r0[:-1]])
        starts = int(np.sum(vis0 & ((np.arange(32) == 0) | (prev != r0))))
        for row in rows:
            vis = row[row != NO_PIXEL]
            total += vis.size if starts > MAX_RUNS else np.unique(vis).size
    return total


def _cases(oracle):
    # about 8 points per covered pixel, so rows of neighbouring points share pixels
    sphere = scenes.sphere_plane(20_011, seed=3).numpy()
    m = scenes.camera((0, 0, 4), (0, 0, 0), (0, 1, 0), 80, 60)
    morton = oracle.gather(sphere, oracle.reorder(sphere, 5, oracle.MORTON))
    shuffled = oracle.gather(sphere, oracle.reorder(sphere, 5, oracle.SHUFFLE))
    return [("morton", morton, m, 80, 60), ("shuffled", shuffled, m, 80, 60), ("original", sphere, m, 80, 60)]


def test_dedup_sends_one_atomic_per_distinct_pixel_per_warp_row(dbg, oracle):
    for name, pts, m, W, H in _cases(oracle):
        dbg.setup(pts, m, W, H)
        pix = _pixels(oracle, pts, m, W, H)
        visible = int(np.sum(pix != NO_PIXEL))
        expect_keys = oracle.render_basic(pts, m, W, H)
        keys, cnt = dbg.render_basic(pcr.PCR_VARIANT_DEDUP)
        assert np.array_equal(keys, expect_keys), name
        assert cnt[0] == _expected_dedup_writes(pix), name
        assert cnt[3] == 0, name  # no early reads without the early test
        keys, cnt = dbg.render_basic(pcr.PCR_VARIANT_ATOMICMIN)
        assert np.array_equal(keys, expect_keys) and cnt[0] == visible, name  # one atomic per visible point
        keys, cnt = dbg.render_basic(pcr.PCR_VARIANT_EARLYZ)
        assert np.array_equal(keys, expect_keys), name
        assert cnt[3] == visible and cnt[0] <= visible, name  # every visible point reads first
        if name == "morton":
            # coherent order: deduplication removes a large share of the atomics
            assert _expected_dedup_writes(pix) < 0.6 * visible
        assert dbg.error_word() == 0, name


def test_debug_build_equals_release_and_its_bounds_checks_stay_silent(dbg, oracle):
    for name, pts, m, W, H in _cases(oracle):
        dbg.setup(pts, m, W, H)
        expect_keys = oracle.render_basic(pts, m, W, H)
        for v in pcr.EXACT_VARIANTS:
            keys, _ = dbg.render_basic(v)
            assert np.array_equal(keys, expect_keys), (name, v)
        expect_hq = oracle.render_hq(pts, m, W, H, 1.01)
        pix = _pixels(oracle, pts, m, W, H)
        for v in (pcr.PCR_VARIANT_ATOMICMIN, pcr.PCR_VARIANT_EARLYZ, pcr.PCR_VARIANT_DEDUP_EARLYZ):
            got, cnt = dbg.render_hq(v)
            for a, b in zip(got, expect_hq):
                assert np.array_equal(a, b), (name, v)
            if v == pcr.PCR_VARIANT_ATOMICMIN:
                # one depth atomic and one pair of colour adds per contributing point
                assert cnt[1] == int(np.sum(pix != NO_PIXEL)), name
                contributing = int(np.sum(expect_hq[2] & np.uint64(0xFFFFFFFF)))
                assert cnt[2] == contributing, name
            else:
                assert cnt[2] <= int(np.sum(expect_hq[2] & np.uint64(0xFFFFFFFF))), (name, v)
        assert dbg.error_word() == 0, name


def test_release_build_has_no_counters(request):
    if request.config.getoption("--pcr-debug-build"):
        pytest.skip("the binding runs the debug build (--pcr-debug-build)")
    from gpu_helpers import ensure_built
    ensure_built()
    with pcr.Context(0, stream=torch.cuda.current_stream()) as ctx:
        out = (C.c_uint64 * 4)()
        assert pcr.lib().pcr_debug_counters(ctx.handle, out) == pcr.PCR_ERR_UNSUPPORTED


@pytest.fixture()
def debug_lib():
    """pcr's wrappers bound to the debug library for one test."""
    build.build(debug=True)
    saved = pcr._lib
    pcr._lib = pcr.load_library(pcr.DEBUG_LIB_PATH)
    try:
        yield pcr._lib
    finally:
        pcr._lib = saved


def test_debug_reorder_and_batch_match_the_oracle_with_silent_checks(debug_lib, oracle):
    """The debug build's range checks in the reorder gathers and scatter and
    its pixel checks in the batch phases stay silent on correct inputs, and
    the results are the oracle's."""
    from gpu_helpers import reorder_gpu
    with pcr.Context(0, stream=torch.cuda.current_stream()) as c:
        for n in (1, 6145, 100_003):
            cloud = scenes.random_cloud(n, seed=n + 11).numpy()
            for mode in (pcr.PCR_ORDER_MORTON, pcr.PCR_ORDER_MORTON_SHUFFLE128, pcr.PCR_ORDER_SHUFFLE,
                         pcr.PCR_ORDER_MORTON63, pcr.PCR_ORDER_MORTON63_SHUFFLE128):
                expect = oracle.reorder(cloud, 99 + n, mode)
                dev = torch.from_numpy(cloud.copy()).cuda()
                perm = reorder_gpu(c.handle, dev, 99 + n, mode)
                assert np.array_equal(perm, expect), (n, mode)
                assert np.array_equal(dev.cpu().numpy(), oracle.gather(cloud, expect)), (n, mode)
        assert pcr.pcr_last_device_error(c.handle) == 0
        # a batch: two clouds, views sharing passes, one alone in its pass
        sphere = scenes.sphere_plane(20_011, seed=3).numpy()
        rnd = scenes.random_cloud(3001, seed=4).numpy()
        clouds = [sphere, rnd]
        views = [(0, scenes.camera((0, 0, 4), (0, 0, 0), (0, 1, 0), 80, 60), 80, 60, 3),
                 (0, scenes.camera((1.5, 2.5, 2.0), (0, 0, 0), (0, 0, 1), 64, 48), 64, 48, 2),
                 (1, scenes.camera((0.2, -2.6, 1.4), (0, 0, 0), (0, 0, 1), 40, 30), 40, 30, 1)]
        dev = [torch.from_numpy(x.copy()).cuda() for x in clouds]
        bufs, vs = [], []
        for (ci, m, W, H, flags) in views:
            b = pcr.alloc_framebuffer(W, H, "cuda")
            b["hq_image"] = torch.empty(W * H, dtype=torch.int32, device="cuda")
            bufs.append(b)
            kw = {}
            if flags & pcr.PCR_BATCH_BASIC:
                kw.update(keys=b["keys"], image=b["image"])
            if flags & pcr.PCR_BATCH_HQ:
                kw.update(hq_depth=b["hq_depth"], hq_rg=b["hq_rg"], hq_ba=b["hq_ba"], hq_image=b["hq_image"])
            vs.append(pcr.batch_view(m, W, H, ci, flags, **kw))
        ws = torch.empty(pcr.pcr_batch_workspace_size(), dtype=torch.uint8, device="cuda")
        pcr.pcr_batch_prepare(c.handle, [pcr.batch_cloud(d) for d in dev], vs, 1.01, 0, ws)
        for config in (0, 8):
            pcr.pcr_batch_launch(c.handle, ws, config)
            torch.cuda.synchronize()
            for (ci, m, W, H, flags), b in zip(views, bufs):
                if flags & pcr.PCR_BATCH_BASIC:
                    want = oracle.render_basic(clouds[ci], m, W, H)
                    assert np.array_equal(b["keys"].cpu().numpy().view(np.uint64), want), config
                if flags & pcr.PCR_BATCH_HQ:
                    d, rg, ba = oracle.render_hq(clouds[ci], m, W, H, 1.01)
                    assert np.array_equal(b["hq_rg"].cpu().numpy().view(np.uint64), rg), config
                    assert np.array_equal(b["hq_ba"].cpu().numpy().view(np.uint64), ba), config
        assert pcr.pcr_last_device_error(c.handle) == 0
