"""Batched rendering (many clouds x views in one launch sequence or one CUDA
graph) against the CPU oracle, bit for bit, for every launch configuration."""
import json

import numpy as np
import pytest
import torch

import constructed as cs
from gpu_helpers import ensure_built
from paper_2104_07526_gb300 import pcr, scenes
from random_inputs import random_cloud, random_matrix

pytestmark = pytest.mark.gpu

BASIC, HQ = pcr.PCR_BATCH_BASIC, pcr.PCR_BATCH_HQ
BG = 0x20304050


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    ensure_built()
    c = pcr.Context(0, stream=torch.cuda.current_stream())
    yield c.handle
    c.close()


def _buffers(W, H):
    npx = W * H
    return {"keys": torch.empty(npx, dtype=torch.int64, device="cuda"),
            "image": torch.empty(npx, dtype=torch.int32, device="cuda"),
            "hq_depth": torch.empty(npx, dtype=torch.int32, device="cuda"),
            "hq_rg": torch.empty(npx, dtype=torch.int64, device="cuda"),
            "hq_ba": torch.empty(npx, dtype=torch.int64, device="cuda"),
            "hq_image": torch.empty(npx, dtype=torch.int32, device="cuda")}


def _make_batch():
    """Three clouds (one ragged, one scanline-ordered, one constructed) and
    eight views of mixed size, flags and cameras."""
    rng = np.random.default_rng(31)
    c0 = scenes.random_cloud(1003, seed=1).numpy()
    c1 = scenes.sphere_plane(50_003, seed=2).numpy()
    c2, _, _ = cs.hq_scene(rng, npix=2000)
    clouds = [c0, c1, c2]
    views = [  # (cloud, matrix, W, H, flags)
        (1, scenes.camera((0, 0, 4), (0, 0, 0), (0, 1, 0), 160, 120), 160, 120, BASIC | HQ),
        (0, scenes.camera((0.2, -2.6, 1.4), (0, 0, 0), (0, 0, 1), 64, 48), 64, 48, BASIC),
        (2, cs.camera(), cs.W, cs.H, BASIC | HQ),
        (1, scenes.camera((1.5, 2.5, 2.0), (0, 0, 0), (0, 0, 1), 333, 77), 333, 77, HQ),
        (0, scenes.camera((0.2, -2.6, 1.4), (0, 0, 0), (0, 0, 1), 40, 30), 40, 30, HQ),
        (1, scenes.camera((0, 0, 4), (0, 0, 0), (0, 1, 0), 1, 1), 1, 1, BASIC | HQ),
        (2, cs.camera(), 320, 240, BASIC),
        (1, scenes.camera((-3.0, 0.5, 0.5), (0, 0, 0), (0, 0, 1), 96, 96), 96, 96, BASIC | HQ),
    ]
    return clouds, views


def _expected(oracle, clouds, views):
    out = []
    for c, m, W, H, flags in views:
        e = {}
        if flags & BASIC:
            k = oracle.render_basic(clouds[c], m, W, H)
            e["keys"] = k
            e["image"] = oracle.resolve_basic(k, clouds[c], BG)
        if flags & HQ:
            d, rg, ba = oracle.render_hq(clouds[c], m, W, H, 1.01)
            e.update(hq_depth=d, hq_rg=rg, hq_ba=ba, hq_image=oracle.resolve_hq(rg, ba, BG))
        out.append(e)
    return out


_VIEWS = {"keys": np.uint64, "image": np.uint32, "hq_depth": np.uint32, "hq_rg": np.uint64, "hq_ba": np.uint64,
          "hq_image": np.uint32}


def _check(bufs, expected, tag):
    torch.cuda.synchronize()
    for i, (b, e) in enumerate(zip(bufs, expected)):
        for name, want in e.items():
            got = b[name].cpu().numpy().view(_VIEWS[name])
            assert np.array_equal(got, want), (tag, i, name)


def _prepare(ctx, clouds, views):
    dev = [torch.from_numpy(c.copy()).cuda() if c.shape[0] else None for c in clouds]
    bufs = [_buffers(W, H) for (_, _, W, H, _) in views]
    vs = []
    for (c, m, W, H, flags), b in zip(views, bufs):
        kw = {}
        if flags & BASIC:
            kw.update(keys=b["keys"], image=b["image"])
        if flags & HQ:
            kw.update(hq_depth=b["hq_depth"], hq_rg=b["hq_rg"], hq_ba=b["hq_ba"], hq_image=b["hq_image"])
        vs.append(pcr.batch_view(m, W, H, c, flags, **kw))
    ws = torch.empty(pcr.pcr_batch_workspace_size(), dtype=torch.uint8, device="cuda")
    pcr.pcr_batch_prepare(ctx, [pcr.batch_cloud(d) for d in dev], vs, 1.01, BG, ws)
    return dev, bufs, ws


def _poison(bufs):
    for b in bufs:
        for t in b.values():
            t.fill_(0x5A5A5A5A)


def test_batch_every_config_and_graph(ctx, oracle):
    clouds, views = _make_batch()
    expected = _expected(oracle, clouds, views)
    dev, bufs, ws = _prepare(ctx, clouds, views)
    for config in range(pcr.pcr_batch_num_configs()):
        _poison(bufs)
        pcr.pcr_batch_launch(ctx, ws, config)
        _check(bufs, expected, f"config {config}")
    best = pcr.pcr_batch_autotune(ctx, ws)
    assert 0 <= best < pcr.pcr_batch_num_configs()
    _check(bufs, expected, "autotune")
    g = pcr.pcr_batch_capture(ctx, ws, best)
    try:
        for rep in range(2):
            _poison(bufs)
            pcr.pcr_graph_launch(ctx, g)
            _check(bufs, expected, f"graph {rep}")
    finally:
        pcr.pcr_graph_destroy(g)


def test_batch_empty_cloud_and_single_view(ctx, oracle):
    clouds = [np.zeros((0, 4), np.int32), scenes.random_cloud(129, seed=5).numpy()]
    views = [(0, np.eye(4, dtype=np.float32), 8, 8, BASIC | HQ),
             (1, scenes.camera((0.2, -2.6, 1.4), (0, 0, 0), (0, 0, 1), 16, 16), 16, 16, BASIC | HQ)]
    expected = _expected(oracle, clouds, views)
    dev, bufs, ws = _prepare(ctx, clouds, views)
    _poison(bufs)
    pcr.pcr_batch_launch(ctx, ws, 0)
    _check(bufs, expected, "empty")


def test_batch_rejects_bad_descriptions(ctx):
    cloud = torch.zeros((10, 4), dtype=torch.int32, device="cuda")
    b = _buffers(4, 4)
    ws = torch.empty(pcr.pcr_batch_workspace_size(), dtype=torch.uint8, device="cuda")
    good = dict(keys=b["keys"], image=b["image"])
    m = np.eye(4, dtype=np.float32)
    cases = [
        ([pcr.batch_cloud(cloud)], [pcr.batch_view(m, 4, 4, 1, BASIC, **good)], pcr.PCR_ERR_ARG),  # bad cloud index
        ([pcr.batch_cloud(cloud)], [pcr.batch_view(m, 0, 4, 0, BASIC, **good)], pcr.PCR_ERR_ARG),  # bad size
        ([pcr.batch_cloud(cloud)], [pcr.batch_view(m, 4, 4, 0, 4, **good)], pcr.PCR_ERR_ARG),  # bad flags
        ([pcr.batch_cloud(cloud)], [pcr.batch_view(m, 4, 4, 0, HQ, **good)], pcr.PCR_ERR_ARG),  # missing HQ buffers
        ([pcr.batch_cloud(cloud)], [], pcr.PCR_ERR_ARG),  # no views
    ]
    for clouds, views, status in cases:
        with pytest.raises(pcr.PcrError) as e:
            pcr.pcr_batch_prepare(ctx, clouds, views, 1.01, 0, ws)
        assert e.value.status == status
    with pytest.raises(pcr.PcrError) as e:
        pcr.pcr_batch_prepare(ctx, [pcr.batch_cloud(cloud)], [pcr.batch_view(m, 4, 4, 0, BASIC, **good)], 1.01, 0,
                              ws[:-256])
    assert e.value.status == pcr.PCR_ERR_WORKSPACE
    with pytest.raises(pcr.PcrError):
        pcr.pcr_batch_launch(ctx, ws, pcr.pcr_batch_num_configs())
    # a launch reads the host copy of the tables its context made: another
    # context has none for this workspace, and launches nothing
    pcr.pcr_batch_prepare(ctx, [pcr.batch_cloud(cloud)], [pcr.batch_view(m, 4, 4, 0, BASIC, **good)], 1.01, 0, ws)
    with pcr.Context(0, stream=torch.cuda.current_stream()) as other:
        for call in (lambda: pcr.pcr_batch_launch(other.handle, ws, 0),
                     lambda: pcr.pcr_batch_capture(other.handle, ws, 0),
                     lambda: pcr.pcr_batch_autotune(other.handle, ws),
                     lambda: pcr.pcr_batch_launch_count(other.handle, ws, 0)):
            with pytest.raises(pcr.PcrError) as e:
                call()
            assert e.value.status == pcr.PCR_ERR_ARG


def test_batch_table_limits(ctx, oracle):
    """The largest batches the tables hold: one cloud seen by 256 views, and
    256 clouds (some empty) with one view each; sizes, flags and cameras
    vary from view to view."""
    rng = np.random.default_rng(77)
    one = [scenes.random_cloud(5003, seed=8).numpy()]
    views = []
    for i in range(pcr.PCR_BATCH_MAX_VIEWS):
        W, H = int(rng.integers(1, 41)), int(rng.integers(1, 31))
        a = rng.uniform(0, 2 * np.pi)
        m = scenes.camera((3 * np.cos(a), 3 * np.sin(a), 1.0), (0, 0, 0), (0, 0, 1), W, H)
        views.append((0, m, W, H, int(rng.choice([BASIC, HQ, BASIC | HQ]))))
    many = [scenes.random_cloud(int(rng.integers(1, 300)), seed=100 + i).numpy() if i % 17 else
            np.zeros((0, 4), np.int32) for i in range(pcr.PCR_BATCH_MAX_CLOUDS)]
    views_many = [(i, views[i][1], views[i][2], views[i][3], views[i][4]) for i in range(pcr.PCR_BATCH_MAX_CLOUDS)]
    for clouds, vs in ((one, views), (many, views_many)):
        expected = _expected(oracle, clouds, vs)
        dev, bufs, ws = _prepare(ctx, clouds, vs)
        if clouds is many:
            # every view is alone with its cloud: one-frame views render single-view
            # in both phases, two-frame views keep one shared phase-1 pass
            live = [f for (c, _, _, _, f) in vs if clouds[c].shape[0]]
            singles0 = sum(1 for f in live if f != BASIC | HQ)
            hq = sum(1 for f in live if f & HQ)
            expect = 2 + (1 if any(f == BASIC | HQ for f in live) else 0) + singles0 + hq
            assert pcr.pcr_batch_launch_count(ctx, ws, 0) == expect
            assert pcr.pcr_batch_launch_count(ctx, ws, 8) == expect
        for config in range(pcr.pcr_batch_num_configs()):
            _poison(bufs)
            pcr.pcr_batch_launch(ctx, ws, config)
            _check(bufs, expected, f"limits config {config}")


def test_batch_tune_chooses_and_caches(ctx, oracle, tmp_path):
    """pcr_batch_tune times every (L2 budget, launch configuration) pair,
    leaves the workspace prepared with the winner, and records it per (GPU,
    batch shape): a second call reads the cache and times nothing.  The
    tuned batch renders the oracle's buffers."""
    clouds, views = _make_batch()
    expected = _expected(oracle, clouds, views)
    dev = [torch.from_numpy(c.copy()).cuda() for c in clouds]
    bufs = [_buffers(W, H) for (_, _, W, H, _) in views]
    vs = []
    for (c, m, W, H, flags), b in zip(views, bufs):
        kw = {}
        if flags & BASIC:
            kw.update(keys=b["keys"], image=b["image"])
        if flags & HQ:
            kw.update(hq_depth=b["hq_depth"], hq_rg=b["hq_rg"], hq_ba=b["hq_ba"], hq_image=b["hq_image"])
        vs.append(pcr.batch_view(m, W, H, c, flags, **kw))
    cs_ = [pcr.batch_cloud(d) for d in dev]
    ws = torch.empty(pcr.pcr_batch_workspace_size(), dtype=torch.uint8, device="cuda")
    cache = str(tmp_path / "batch_tuning.jsonl")
    first = pcr.pcr_batch_tune(ctx, cs_, vs, 1.01, BG, ws, cache)
    assert first["from_cache"] == 0 and first["tried"] == 3 * pcr.pcr_batch_num_configs()
    assert first["l2_budget_mb"] in (64, 96, 128) and 0 <= first["config"] < pcr.pcr_batch_num_configs()
    assert first["threads"] in (256, 512) and first["unroll1"] in (2, 4) and first["unroll2"] in (2, 4)
    assert first["single_colors"] == (first["config"] >> 3) & 1
    assert 0 < first["best_ms"] <= first["default_ms"]
    _poison(bufs)
    pcr.pcr_batch_launch(ctx, ws, first["config"])
    _check(bufs, expected, "tuned")
    # lines it cannot use are skipped: garbage, and entries for this GPU and
    # shape with a budget or configuration it does not offer
    with open(cache) as f:
        line = f.read().splitlines()[0]
    entry = json.loads(line)
    with open(cache, "a") as f:
        f.write("not json at all\n")
        f.write(json.dumps({**entry, "budget_mb": 77}) + "\n")
        f.write(json.dumps({**entry, "config": 99}) + "\n")
    again = pcr.pcr_batch_tune(ctx, cs_, vs, 1.01, BG, ws, cache)
    assert again["from_cache"] == 1 and again["tried"] == 0
    assert (again["l2_budget_mb"], again["config"]) == (first["l2_budget_mb"], first["config"])
    _poison(bufs)
    pcr.pcr_batch_launch(ctx, ws, again["config"])
    _check(bufs, expected, "from cache")
    with open(cache) as f:
        lines = f.read().splitlines()
    assert len(lines) == 4 and '"budget_mb": %d' % first["l2_budget_mb"] in lines[0]
    # another shape misses the cache
    other = pcr.pcr_batch_tune(ctx, cs_, vs[:3], 1.01, BG, ws, cache)
    assert other["from_cache"] == 0


@pytest.mark.parametrize("seed", range(8))
def test_batch_random_descriptions(ctx, oracle, seed):
    """Seeded random batches: 1-6 clouds of 0-20000 points, 1-24 views with
    random clouds, flags, cameras and sizes (a few large enough that a
    cloud's views need several passes, and clouds with a single view, which
    take the single-view kernels), in a random launch configuration; every
    buffer of every view against the oracle."""
    rng = np.random.default_rng(3000 + seed)
    clouds = []
    for _ in range(int(rng.integers(1, 7))):
        c = random_cloud(rng)
        clouds.append(c[: int(rng.integers(0, c.shape[0] + 1))] if rng.random() < 0.2 else c)
    views = []
    for _ in range(int(rng.integers(1, 25))):
        c = int(rng.integers(0, len(clouds)))
        if rng.random() < 0.15:
            W, H = int(rng.integers(1500, 2600)), int(rng.integers(1500, 2600))
        else:
            W, H = int(rng.integers(1, 200)), int(rng.integers(1, 200))
        flags = (BASIC, HQ, BASIC | HQ)[int(rng.integers(0, 3))]
        cloud = clouds[c] if clouds[c].shape[0] else np.zeros((1, 4), np.int32)
        views.append((c, random_matrix(rng, cloud, W, H), W, H, flags))
    expected = _expected(oracle, clouds, views)
    dev, bufs, ws = _prepare(ctx, clouds, views)
    config = int(rng.integers(0, pcr.pcr_batch_num_configs()))
    _poison(bufs)
    pcr.pcr_batch_launch(ctx, ws, config)
    _check(bufs, expected, f"seed {seed} config {config}")
