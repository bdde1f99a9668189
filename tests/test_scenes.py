"""The seeded synthetic inputs: each scene matches the recipe the benchmark
states, depends on its seed and on each point's index alone, and is the same
on every call.  These inputs stand in for the paper's datasets (Sec. 5),
which are not available here."""
import math

import numpy as np
import torch

from paper_2104_07526_gb300 import scenes


def _xyz(cloud: torch.Tensor) -> np.ndarray:
    return cloud[:, :3].contiguous().view(torch.float32).numpy().astype(np.float64)


def _rgba(cloud: torch.Tensor) -> np.ndarray:
    return cloud[:, 3].contiguous().numpy().view(np.uint32)


def test_generators_are_deterministic_and_seeded():
    for make in (lambda s: scenes.random_cloud(5000, seed=s), lambda s: scenes.sphere_plane(5000, seed=s),
                 lambda s: scenes.boxes(5000, seed=s), lambda s: scenes.scan(5000, seed=s)):
        a, b, c = make(0), make(0), make(1)
        assert torch.equal(a, b)
        assert not torch.equal(a, c)


def test_scan_points_depend_on_their_index_alone():
    """The CPU baseline renders a strided sample of the 800M cloud made
    point by point; it must hold the same bytes as the full cloud."""
    n = 200_003
    full = scenes.scan(n, seed=0)
    rng = np.random.default_rng(5)
    idx = torch.from_numpy(np.sort(rng.choice(n, size=5000, replace=False)).astype(np.int64))
    assert torch.equal(scenes.scan(n, seed=0, indices=idx), full[idx])
    assert torch.equal(scenes.scan(n, seed=0, chunk=4096), full)  # chunking changes nothing


def test_sphere_plane_recipe():
    n = 10_000
    xyz = _xyz(scenes.sphere_plane(n, seed=0))
    r = np.linalg.norm(xyz[: n // 2], axis=1)
    assert np.allclose(r, 1.0, atol=1e-5)  # the first half on the unit sphere
    plane = xyz[n // 2:]
    assert np.all(plane[:, 2] == -1.0) and np.all(np.abs(plane[:, :2]) <= 2.0)


def test_boxes_recipe():
    n = 100_000
    cloud = scenes.boxes(n, seed=3)
    xyz, rgba = _xyz(cloud), _rgba(cloud)
    assert np.all(np.isfinite(xyz)) and np.all(rgba >> 24 == 255)
    assert np.all(np.abs(xyz[:, :2]) <= 50.0 + 2.5 + 1e-3)  # centres in [-50, 50]^2, half sides up to 2.5
    assert np.all(xyz[:, 2] >= -1e-3) and np.all(xyz[:, 2] <= 5.0 + 1e-3)
    layout = scenes.boxes_layout(3)
    assert layout.centres.shape == (200, 2) and np.all((layout.sides >= 0.1) & (layout.sides <= 5.0))
    # points per face follow the face areas, and the counts add up to n
    origin, u, v, rgb, area = scenes._box_faces(layout)
    counts = scenes._counts_by_area(n, area)
    assert counts.sum() == n and np.all(np.abs(counts - area / area.sum() * n) <= len(area))
    ground = xyz[-counts[-1]:]  # the ground is the last face, grey
    assert np.all(np.abs(ground[:, 2]) <= 1e-3) and np.all(_rgba(cloud[-counts[-1]:]) & 0xFFFFFF == 0x808080)


def test_scan_recipe():
    n = 200_000
    xyz = _xyz(scenes.scan(n, seed=0))
    lay = scenes.scan_layout(n, 0)
    nfac = int(lay.wall_counts.sum())
    assert nfac == int(0.6 * n) and lay.walls.shape == (40, 6)
    w, h = lay.walls[:, 3], lay.walls[:, 4]
    assert np.all((w >= 10) & (w <= 60) & (h >= 5) & (h <= 30))
    assert np.all(np.isfinite(xyz))
    # the terrain comes in row scanlines: x grows along each row
    ter = xyz[nfac:]
    assert np.all(np.abs(ter[:, :2]) <= 200.0 + 1e-3)
    rows = ter[: lay.terrain_cols * 4]
    assert np.all(np.diff(rows[: lay.terrain_cols, 0]) > 0)  # one row sweeps x


def test_cameras_and_batch_views():
    views = scenes.batch_views(8)
    assert len(views) == 64
    sizes = sorted({v.width for _, v in views})
    assert sizes == list(scenes.BATCH_VIEW_SIZES) and all(v.width == v.height for _, v in views)
    assert [c for c, _ in views] == [c for c in range(8) for _ in range(8)]
    # a camera maps its target to the screen centre, in front of the eye
    m = scenes.camera((0.0, -10.0, 5.0), (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), 640, 480).astype(np.float64)
    clip = m @ np.array([0.0, 0.0, 0.0, 1.0])
    assert clip[3] > 0 and abs(clip[0] / clip[3]) < 1e-6 and abs(clip[1] / clip[3]) < 1e-6
    assert abs(clip[3] - math.sqrt(125.0)) < 1e-4  # w is the distance along the view axis


def test_serve_requests_recipe():
    reqs = scenes.serve_requests(4000, 2000.0, seed=7, num_clouds=16)
    again = scenes.serve_requests(4000, 2000.0, seed=7, num_clouds=16)
    assert all(a[:2] == b[:2] and a[3:] == b[3:] and np.array_equal(a[2], b[2]) for a, b in zip(reqs, again))
    t = np.array([r[0] for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(t[-1] - 2.0) < 0.15  # 4000 arrivals at 2000/s span about 2 s
    assert {(r[3], r[4]) for r in reqs} == set(scenes.SERVE_RESOLUTIONS)
    assert {r[1] for r in reqs} == set(range(16))
    basic = sum(r[5] == 1 for r in reqs) / len(reqs)
    assert 0.45 < basic < 0.55 and {r[5] for r in reqs} == {1, 2}
    sizes = scenes.SERVE_CLOUD_SIZES
    assert len(sizes) == 16 and sizes[0] == 1_000_000 and sizes[-1] == 300_000_000
