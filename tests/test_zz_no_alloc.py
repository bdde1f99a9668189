"""The allocation-free reorder (pcr_reorder_morton_shuffle128_noalloc).

It serves callers that cannot allocate device memory for a workspace (a
plugin handed only the point buffer, code under another allocator's pool, a
frame loop that must not synchronise the device).  Its output must equal the
workspace entry point's, bit for bit, on consecutive calls that reuse the
library's one scratch array.  This file is collected last and is
self-contained, so it passes alone in a fresh process or after the rest.
"""
import numpy as np
import pytest
import torch

from paper_2104_07526_gb300 import build, pcr, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    c = pcr.Context(0, stream=torch.cuda.current_stream())
    yield c.handle
    c.close()


def _with_workspace(h, cloud, seed, mode):
    n = cloud.shape[0]
    pts = cloud.clone()
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    ws = torch.empty(pcr.pcr_reorder_workspace_size(n), dtype=torch.uint8, device="cuda")
    pcr.pcr_reorder_morton_shuffle128(h, pts, n, seed, mode, ws, perm)
    return pts, perm


def _without_workspace(h, cloud, seed, mode):
    n = cloud.shape[0]
    pts = cloud.clone()
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    pcr.pcr_reorder_morton_shuffle128_noalloc(h, pts, n, seed, mode, perm)
    return pts, perm


def test_noalloc_matches_workspace_entry_on_consecutive_calls(ctx):
    """Two calls in a row share the scratch array; each must match the
    workspace entry point exactly (points and permutation)."""
    full = pcr.PCR_REORDER_NOALLOC_MAX_POINTS
    cases = [
        (scenes.scan(200_003, seed=3).cuda(), 0xABC, pcr.PCR_ORDER_MORTON_SHUFFLE128),
        (scenes.random_cloud(full, seed=4).cuda(), 0xDEF, pcr.PCR_ORDER_MORTON),
        (scenes.sphere_plane(1000, seed=5).cuda(), 7, pcr.PCR_ORDER_SHUFFLE),
        # the 63-bit orders keep their high code words in the part of the
        # array a 30-bit call used for its record copy, right after one
        (scenes.random_cloud(full, seed=8).cuda(), 0x63, pcr.PCR_ORDER_MORTON63),
        (scenes.scan(70_001, seed=9).cuda(), 0x31, pcr.PCR_ORDER_MORTON),
        (scenes.scan(130_000, seed=10).cuda(), 0x64, pcr.PCR_ORDER_MORTON63_SHUFFLE128),
    ]
    for cloud, seed, mode in cases:
        a_pts, a_perm = _with_workspace(ctx, cloud, seed, mode)
        b_pts, b_perm = _without_workspace(ctx, cloud, seed, mode)
        torch.cuda.synchronize()
        assert torch.equal(a_perm, b_perm), mode
        assert torch.equal(a_pts, b_pts), mode
        assert not torch.equal(b_pts, cloud)  # the order did change


def test_noalloc_rejects_clouds_beyond_its_limit(ctx):
    n = pcr.PCR_REORDER_NOALLOC_MAX_POINTS + 1
    cloud = scenes.random_cloud(n, seed=6).cuda()
    before = cloud.clone()
    with pytest.raises(pcr.PcrError) as e:
        pcr.pcr_reorder_morton_shuffle128_noalloc(ctx, cloud, n, 1, pcr.PCR_ORDER_MORTON)
    assert e.value.status == pcr.PCR_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert torch.equal(cloud, before)  # nothing was launched


def test_noalloc_takes_no_device_memory(ctx):
    """After a warm-up call (which may load the library's device code), calls
    leave the device's free memory unchanged."""
    n = 100_000
    cloud = scenes.scan(n, seed=11).cuda()
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    pts = cloud.clone()
    pcr.pcr_reorder_morton_shuffle128_noalloc(ctx, pts, n, 1, pcr.PCR_ORDER_MORTON_SHUFFLE128, perm)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for mode in (pcr.PCR_ORDER_MORTON_SHUFFLE128, pcr.PCR_ORDER_MORTON, pcr.PCR_ORDER_SHUFFLE,
                 pcr.PCR_ORDER_MORTON63, pcr.PCR_ORDER_MORTON63_SHUFFLE128):
        pcr.pcr_reorder_morton_shuffle128_noalloc(ctx, pts, n, 2, mode, perm)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
