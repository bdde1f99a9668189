"""GPU parity for the colour-payload key (Sec. 3.1, the key as Listing "basic"
prints it) and the busy-loop comparison kernel (Sec. 2 and Sec. 5), against
the CPU oracle, bit for bit.

The busy-loop's lock wait is bounded; one test makes it run out on purpose by
handing the kernel lock words that are already held and that nothing
releases, and checks the status the kernel reports.
"""
import numpy as np
import pytest
import torch

import constructed as cs
from gpu_helpers import Renderer, U64_EMPTY
from paper_2104_07526_gb300 import pcr, scenes

pytestmark = pytest.mark.gpu

EXACT = pcr.EXACT_VARIANTS
BUSY = pcr.PCR_VARIANT_BUSY_LOOP


@pytest.fixture(scope="module")
def r():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    rend = Renderer()
    yield rend
    rend.close()


@pytest.fixture(scope="module")
def sphere():
    return scenes.sphere_plane(200_003, seed=0).numpy()


# --- colour payload -------------------------------------------------------------

def test_rgb_all_variants(r, oracle, sphere):
    view = scenes.sphere_plane_views()[0]
    expect = oracle.render_rgb(sphere, view.matrix, view.width, view.height)
    img_expect = oracle.resolve_rgb(expect, 0x0A0B0C0D)
    assert (expect != U64_EMPTY).sum() > 10000
    r.upload(sphere)
    r.view(view.matrix, view.width, view.height)
    for v in EXACT:
        assert np.array_equal(r.render_rgb(v), expect), pcr.VARIANT_NAMES[v]
        assert np.array_equal(r.resolve(pcr.PCR_RESOLVE_RGB, 0x0A0B0C0D), img_expect), pcr.VARIANT_NAMES[v]


def test_rgb_depth_and_colour_ties(r, oracle):
    """One pixel, many points: random depths with random colours, then one
    depth with colours drawn from a few values (many exact key ties), then
    identical keys everywhere (the pairwise reduction must keep one)."""
    n = 200_000
    rng = np.random.default_rng(8)
    m = cs.camera()
    r.view(m, cs.W, cs.H)
    d = rng.integers(4, 4000, size=n) / 256.0
    scenes_ = [
        (np.stack([np.zeros(n), np.zeros(n), cs.EYE_Z - d], 1), rng.integers(0, 1 << 32, size=n, dtype=np.uint64)),
        (np.tile([[0.0, 0.0, 1.5]], (n, 1)), rng.choice([0xFF00FF00, 0x00123456, 0xFF000102, 0x7F000102], size=n)),
        (np.tile([[0.0, 0.0, 1.5]], (n, 1)), np.full(n, 0xFF332211, dtype=np.uint64)),
    ]
    for xyz, rgba in scenes_:
        cloud = cs.pack(xyz, rgba.astype(np.uint32))
        expect = oracle.render_rgb(cloud, m, cs.W, cs.H)
        r.upload(cloud)
        for v in EXACT:
            assert np.array_equal(r.render_rgb(v), expect), pcr.VARIANT_NAMES[v]


def test_rgb_constructed_and_ragged(r, oracle):
    rng = np.random.default_rng(23)
    cloud, _, _, _ = cs.depth_scene(rng, npix=3000, max_per_pixel=8)
    expect = oracle.render_rgb(cloud, cs.camera(), cs.W, cs.H)
    r.upload(cloud)
    r.view(cs.camera(), cs.W, cs.H)
    for v in EXACT:
        assert np.array_equal(r.render_rgb(v), expect), pcr.VARIANT_NAMES[v]
    m = scenes.camera((0.2, -2.6, 1.4), (0, 0, 0), (0, 0, 1), 32, 24)
    r.view(m, 32, 24)
    for n in (0, 1, 33, 129, 4097):
        small = scenes.random_cloud(n, seed=n + 300).numpy() if n else np.zeros((0, 4), np.int32)
        expect = oracle.render_rgb(small, m, 32, 24)
        r.upload(small)
        for v in EXACT:
            assert np.array_equal(r.render_rgb(v), expect), (n, pcr.VARIANT_NAMES[v])


def test_rgb_just_set_writes_valid_keys(r, oracle, sphere):
    view = scenes.sphere_plane_views()[0]
    expect = oracle.render_rgb(sphere, view.matrix, view.width, view.height)
    r.upload(sphere)
    r.view(view.matrix, view.width, view.height)
    got = r.render_rgb(pcr.PCR_VARIANT_JUST_SET)
    assert np.array_equal(got == U64_EMPTY, expect == U64_EMPTY)
    # every written key is the colour key of some point landing on its pixel
    offered = {}
    p = np.ascontiguousarray(sphere[:, :3]).view(np.float32)
    rgba = sphere[:, 3].view(np.uint32)
    for i in range(sphere.shape[0]):
        hit = oracle.project(view.matrix, view.width, view.height, *p[i])
        if hit is not None:
            offered.setdefault(hit[0], set()).add(oracle.key_rgb(hit[1], int(rgba[i])))
    hit = np.nonzero(got != U64_EMPTY)[0]
    assert len(hit) == len(offered)
    for j in hit:
        assert int(got[j]) in offered[int(j)]


# --- busy-loop -------------------------------------------------------------------

def test_busy_loop_matches_atomic_render(r, oracle, sphere):
    """The lock-protected update keeps the smaller (depth, index) key, so the
    buffer equals the atomicMin render's."""
    view = scenes.sphere_plane_views()[0]
    expect = oracle.render_basic(sphere, view.matrix, view.width, view.height)
    r.upload(sphere)
    r.view(view.matrix, view.width, view.height)
    assert pcr.pcr_last_device_error(r.h) == 0
    for _ in range(2):
        assert np.array_equal(r.render_basic(BUSY), expect)
    assert pcr.pcr_last_device_error(r.h) == 0
    assert int(r.fb["locks"].abs().sum()) == 0  # every lock given back


def test_busy_loop_contention_and_ties(r, oracle):
    """Many points on one pixel, distinct depths, then one depth (the
    smallest index must win), with a generous wait limit."""
    n = 50_000
    rng = np.random.default_rng(6)
    m = cs.camera()
    r.view(m, cs.W, cs.H)
    pcr.pcr_set_lock_buffer(r.h, r.fb["locks"], 2_000_000)
    try:
        d = rng.integers(4, 4000, size=n) / 256.0
        for xyz in (np.stack([np.zeros(n), np.zeros(n), cs.EYE_Z - d], 1), np.tile([[0.0, 0.0, 1.5]], (n, 1))):
            cloud = cs.pack(xyz, np.arange(n, dtype=np.uint32))
            expect = oracle.render_basic(cloud, m, cs.W, cs.H)
            r.upload(cloud)
            assert np.array_equal(r.render_basic(BUSY), expect)
        rng2 = np.random.default_rng(7)
        cloud, expected, _, _ = cs.depth_scene(rng2, npix=3000, max_per_pixel=8)
        r.upload(cloud)
        assert np.array_equal(r.render_basic(BUSY), expected)
        assert pcr.pcr_last_device_error(r.h) == 0
    finally:
        pcr.pcr_set_lock_buffer(r.h, r.fb["locks"], 0)


def test_busy_loop_wait_limit_reports_timeout(r, oracle):
    """Lock words that are held and never released: every wait runs out
    after the limit (2 ms), the kernel ends, the error word carries
    PCR_DEVICE_ERROR_WAIT_TIMEOUT, and the context keeps working."""
    cloud = scenes.random_cloud(20_000, seed=12).numpy()
    m = scenes.camera((0.2, -2.6, 1.4), (0, 0, 0), (0, 0, 1), 64, 48)
    r.upload(cloud)
    r.view(m, 64, 48)
    assert pcr.pcr_last_device_error(r.h) == 0
    held = torch.ones(64 * 48, dtype=torch.int32, device="cuda")
    pcr.pcr_set_lock_buffer(r.h, held, 2000)
    try:
        pcr.pcr_clear(r.h, pcr.PCR_CLEAR_KEYS)
        pcr.pcr_render_basic(r.h, BUSY, False)  # clear=False keeps the held locks
        torch.cuda.synchronize()
        assert pcr.pcr_last_device_error(r.h) == pcr.PCR_DEVICE_ERROR_WAIT_TIMEOUT
        assert torch.all(held == 1)  # the kernel never wrote a lock it did not take
    finally:
        pcr.pcr_set_lock_buffer(r.h, r.fb["locks"], 0)
    expect = oracle.render_basic(cloud, m, 64, 48)
    assert np.array_equal(r.render_basic(BUSY), expect)
    assert np.array_equal(r.render_basic(pcr.PCR_VARIANT_DEDUP_EARLYZ), expect)
    assert pcr.pcr_last_device_error(r.h) == 0


def test_busy_loop_needs_lock_buffer(r):
    r.view(np.eye(4, dtype=np.float32), 8, 8)
    pcr.pcr_set_lock_buffer(r.h, None, 0)
    try:
        with pytest.raises(pcr.PcrError) as e:
            pcr.pcr_render_basic(r.h, BUSY, True)
        assert e.value.status == pcr.PCR_ERR_ARG
        with pytest.raises(pcr.PcrError):
            pcr.pcr_render_rgb(r.h, BUSY, True)
    finally:
        pcr.pcr_set_lock_buffer(r.h, r.fb["locks"], 0)
