"""GPU parity for the vertex orders (Sec. 4, Sec. 5): permutation and
reordered records bit-exact against the oracle; rendering is invariant under
every order."""
import numpy as np
import pytest
import torch

import constructed as cs
from gpu_helpers import Renderer, reorder_gpu, U64_EMPTY
from paper_2104_07526_gb300 import pcr, scenes

pytestmark = pytest.mark.gpu

MODES = (pcr.PCR_ORDER_MORTON, pcr.PCR_ORDER_MORTON_SHUFFLE128, pcr.PCR_ORDER_SHUFFLE, pcr.PCR_ORDER_MORTON63,
         pcr.PCR_ORDER_MORTON63_SHUFFLE128)


@pytest.fixture(scope="module")
def r():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    rend = Renderer()
    yield rend
    rend.close()


@pytest.mark.parametrize("n", [0, 1, 2, 127, 128, 129, 1000, 5119, 5120, 5121, 6143, 6144, 6145, 8191, 8192, 8193,
                               10241, 12289, 100_003])
def test_reorder_matches_oracle(r, oracle, n):
    cloud = scenes.random_cloud(n, seed=n + 7).numpy() if n else np.zeros((0, 4), np.int32)
    for mode in MODES:
        seed = 0xC0FFEE + n
        expect = oracle.reorder(cloud, seed, mode)
        dev = torch.from_numpy(cloud.copy()).cuda() if n else torch.zeros((0, 4), dtype=torch.int32, device="cuda")
        perm = reorder_gpu(r.h, dev, seed, mode)
        assert np.array_equal(perm, expect), (n, mode)
        assert np.array_equal(dev.cpu().numpy(), oracle.gather(cloud, expect) if n else cloud), (n, mode)


@pytest.mark.parametrize("n", [300_017, 5_000_017])
def test_reorder_scene_with_duplicates(r, oracle, n):
    """Scanline scene (many equal Morton codes: stability decides) at sizes
    spanning many sort tiles with a ragged tail; 5M points is 814 tiles, more
    than the scatter kernel keeps resident at once (4 per SM), so tiles run
    in several waves."""
    cloud = scenes.scan(n, seed=1).numpy()
    for mode in MODES:
        expect = oracle.reorder(cloud, 42, mode)
        dev = torch.from_numpy(cloud.copy()).cuda()
        perm = reorder_gpu(r.h, dev, 42, mode)
        assert np.array_equal(perm, expect), mode
    assert pcr.pcr_last_device_error(r.h) == 0


@pytest.mark.parametrize("n", [129, 8193, 100_003])
def test_reorder_without_permutation(r, oracle, n):
    """Without a permutation output the last sort pass takes its other
    record-moving loops; the records must be the same."""
    cloud = scenes.random_cloud(n, seed=n + 3).numpy()
    for mode in MODES:
        expect = oracle.gather(cloud, oracle.reorder(cloud, 99, mode))
        dev = torch.from_numpy(cloud.copy()).cuda()
        ws = torch.empty(pcr.pcr_reorder_workspace_size(n), dtype=torch.uint8, device="cuda")
        pcr.pcr_reorder_morton_shuffle128(r.h, dev, n, 99, mode, ws, None)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy(), expect), (n, mode)


def test_reorder_degenerate_and_nonfinite(r, oracle):
    same = cs.pack(np.tile([[1.0, 2.0, 3.0]], (1000, 1)), np.arange(1000, dtype=np.uint32))
    odd = scenes.random_cloud(3000, seed=4).numpy()
    odd[5, 0] = np.float32(np.nan).view(np.int32)
    odd[9, 1] = np.float32(-0.0).view(np.int32)
    odd[11, 2] = np.float32(np.nan).view(np.int32)
    for cloud in (same, odd):
        for mode in MODES:
            expect = oracle.reorder(cloud, 5, mode)
            dev = torch.from_numpy(cloud.copy()).cuda()
            assert np.array_equal(reorder_gpu(r.h, dev, 5, mode), expect), mode


def test_render_invariant_under_orders(r, oracle):
    """Sec. 4: reordering changes speed, not the image.  Depth halves match
    exactly.  Where several points share the minimum depth (the ground plane
    of this scene is at one depth) the index tie-break may pick another of
    them, so each winner is checked to be a minimum-depth point of its
    pixel; the reordered buffer also matches the oracle bit for bit."""
    cloud = scenes.sphere_plane(120_000, seed=2).numpy()
    view = scenes.sphere_plane_views()[0]
    W, H = view.width, view.height
    base = oracle.render_basic(cloud, view.matrix, W, H)
    hit = np.nonzero(base != U64_EMPTY)[0]
    p = np.ascontiguousarray(cloud[:, :3]).view(np.float32)
    for mode in MODES:
        dev = torch.from_numpy(cloud.copy()).cuda()
        perm = reorder_gpu(r.h, dev, 9, mode).astype(np.int64)
        pcr.pcr_upload_points(r.h, dev, dev.shape[0])
        r.points = dev
        r.view(view.matrix, W, H)
        got = r.render_basic(pcr.PCR_VARIANT_DEDUP_EARLYZ)
        moved = oracle.gather(cloud, perm.astype(np.uint32))
        assert np.array_equal(got, oracle.render_basic(moved, view.matrix, W, H)), mode
        assert np.array_equal(got >> np.uint64(32), base >> np.uint64(32)), mode
        for px in hit[:: max(1, hit.size // 3000)]:
            old = perm[int(got[px]) & 0xFFFFFFFF]
            pr = oracle.project(view.matrix, W, H, *p[old])
            assert pr is not None and pr[0] == px
            assert int(np.float32(pr[1]).view(np.uint32)) == int(base[px]) >> 32
        img = r.resolve(pcr.PCR_RESOLVE_BASIC, 0)
        assert np.array_equal(img, oracle.resolve_basic(got, moved, 0)), mode


def test_reorder_errors(r):
    n = 1000
    dev = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    need = pcr.pcr_reorder_workspace_size(n)
    small = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(pcr.PcrError) as e:
        pcr.pcr_reorder_morton_shuffle128(r.h, dev, n, 0, pcr.PCR_ORDER_MORTON, small)
    assert e.value.status == pcr.PCR_ERR_WORKSPACE
    with pytest.raises(pcr.PcrError) as e:
        pcr.pcr_reorder_morton_shuffle128(r.h, dev, n, 0, pcr.PCR_ORDER_MORTON, None)
    assert e.value.status == pcr.PCR_ERR_WORKSPACE
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(pcr.PcrError) as e:
        pcr.pcr_reorder_morton_shuffle128(r.h, dev, n, 0, 5, ws)
    assert e.value.status == pcr.PCR_ERR_ARG
    with pytest.raises(pcr.PcrError) as e:
        pcr.pcr_reorder_morton_shuffle128(r.h, dev.data_ptr() + 4, n, 0, 0, ws)
    assert e.value.status == pcr.PCR_ERR_ARG
