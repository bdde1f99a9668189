"""Serving loop: continuous batching of view requests over resident clouds.

Every result must equal the request rendered alone (the CPU oracle), bit for
bit, whatever batch it shared; eviction under a small arena must not change
results."""
import time

import numpy as np
import pytest
import torch

import constructed as cs
from gpu_helpers import ensure_built
from paper_2104_07526_gb300 import pcr, scenes
from random_inputs import random_cloud, random_matrix

pytestmark = pytest.mark.gpu

BASIC, HQ = pcr.PCR_BATCH_BASIC, pcr.PCR_BATCH_HQ
BG = 0x01010101


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    ensure_built()
    c = pcr.Context(0, stream=torch.cuda.current_stream())
    yield c.handle
    c.close()


def _download(h, ptr, count, dtype):
    out = np.empty(count, dtype=dtype)
    pcr.pcr_download(h, out, ptr, out.nbytes)
    return out


def _check_result(h, srv, ticket, cloud, m, W, H, flags, oracle):
    res = pcr.pcr_server_get_result(srv, ticket)
    assert (res.width, res.height, res.flags) == (W, H, flags)
    npx = W * H
    if flags & BASIC:
        k = oracle.render_basic(cloud, m, W, H)
        assert np.array_equal(_download(h, res.keys, npx, np.uint64), k)
        assert np.array_equal(_download(h, res.image, npx, np.uint32), oracle.resolve_basic(k, cloud, BG))
    if flags & HQ:
        d, rg, ba = oracle.render_hq(cloud, m, W, H, 1.01)
        assert np.array_equal(_download(h, res.hq_depth, npx, np.uint32), d)
        assert np.array_equal(_download(h, res.hq_rg, npx, np.uint64), rg)
        assert np.array_equal(_download(h, res.hq_ba, npx, np.uint64), ba)
        assert np.array_equal(_download(h, res.hq_image, npx, np.uint32), oracle.resolve_hq(rg, ba, BG))
    assert res.done_us >= res.launch_us >= res.submit_us > 0


def _drain(srv, tickets, on_done=None, timeout_s=60.0):
    """Step until every ticket is done; on_done(ticket) runs (and may
    release the slot) as each one finishes, as a client would."""
    pending = list(tickets)
    t0 = time.time()
    while pending:
        pcr.pcr_server_step(srv)
        still = []
        for t in pending:
            if pcr.pcr_server_state(srv, t) == pcr.PCR_REQUEST_DONE:
                if on_done:
                    on_done(t)
            else:
                still.append(t)
        pending = still
        assert time.time() - t0 < timeout_s, "server did not finish"


def _clouds():
    rng = np.random.default_rng(41)
    hq_cloud, _, _ = cs.hq_scene(rng, npix=1500)
    return [scenes.sphere_plane(60_003, seed=1).numpy(), scenes.random_cloud(7001, seed=2).numpy(), hq_cloud,
            scenes.scan(120_005, seed=3).numpy()]


def _requests(rng, clouds, count, max_w, max_h):
    out = []
    for _ in range(count):
        c = int(rng.integers(0, len(clouds)))
        W = int(rng.integers(1, max_w + 1))
        H = int(rng.integers(1, max_h + 1))
        flags = int(rng.choice([BASIC, HQ, BASIC | HQ]))
        if c == 2:
            m = cs.camera()
        elif c == 3:
            m = scenes.camera((0, -300, 200), (0, 0, 0), (0, 0, 1), W, H)
        else:
            a = rng.uniform(0, 2 * np.pi)
            m = scenes.camera((3 * np.cos(a), 3 * np.sin(a), 1.5), (0, 0, 0), (0, 0, 1), W, H)
        out.append((c, m, W, H, flags))
    return out


def test_mixed_requests_match_rendering_alone(ctx, oracle):
    clouds = _clouds()
    dev = [torch.from_numpy(c.copy()).cuda() for c in clouds]
    arena = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    srv = pcr.pcr_server_create(ctx, arena, 200, 150, num_slots=12, max_batch_views=7, max_inflight=3,
                                background_rgba=BG)
    try:
        host = [np.ascontiguousarray(c) for c in clouds]
        pcr.pcr_server_add_device_cloud(srv, 10, dev[0])
        pcr.pcr_server_add_cloud(srv, 11, host[1])
        pcr.pcr_server_add_device_cloud(srv, 12, dev[2])
        pcr.pcr_server_add_cloud(srv, 13, host[3])
        rng = np.random.default_rng(42)
        reqs = _requests(rng, clouds, 30, 200, 150)
        by_ticket = {}

        def finish(t):
            c, m, W, H, flags = by_ticket.pop(t)
            _check_result(ctx, srv, t, clouds[c], m, W, H, flags, oracle)
            pcr.pcr_server_release(srv, t)

        # submit in waves while earlier requests are still on the GPU
        tickets = []
        for i, req in enumerate(reqs):
            c, m, W, H, flags = req
            t = pcr.pcr_server_submit(srv, 10 + c, m, W, H, flags)
            by_ticket[t] = req
            tickets.append(t)
            if i % 4 == 3:
                pcr.pcr_server_step(srv)
        _drain(srv, tickets, finish)
        assert not by_ticket
        st = pcr.pcr_server_stats_get(srv)
        assert st["completed"] == len(reqs) and st["batches"] >= 3 and st["queued"] == 0
        # the same request alone, in a fresh batch of one, gives the same result
        c, m, W, H, flags = reqs[0]
        t = pcr.pcr_server_submit(srv, 10 + c, m, W, H, flags)
        _drain(srv, [t])
        _check_result(ctx, srv, t, clouds[c], m, W, H, flags, oracle)
        pcr.pcr_server_release(srv, t)
    finally:
        pcr.pcr_server_destroy(srv)


def test_both_launch_paths_match_rendering_alone(ctx, oracle):
    """A batch in which no two views share a cloud shares no pass over a
    cloud's points: the batch launch sends every view through the
    single-view kernels.  Views of one cloud batched together share passes
    through the batch kernels.  One view per batch forces the first path;
    submitting views of one cloud together with room for them all forces the
    second.  Both give the oracle's buffers."""
    clouds = _clouds()
    dev = [torch.from_numpy(c.copy()).cuda() for c in clouds]
    arena = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    rng = np.random.default_rng(43)
    for views_per_batch, same_cloud in ((1, False), (6, True)):
        srv = pcr.pcr_server_create(ctx, arena, 200, 150, num_slots=8, max_batch_views=views_per_batch,
                                    max_inflight=2, background_rgba=BG)
        try:
            for i, d in enumerate(dev):
                pcr.pcr_server_add_device_cloud(srv, i, d)
            reqs = _requests(rng, clouds, 12, 200, 150)
            if same_cloud:
                reqs = [(3, scenes.camera((0, -300, 200), (0, 0, 0), (0, 0, 1), W, H), W, H, f)
                        for _, _, W, H, f in reqs]
            by_ticket = {pcr.pcr_server_submit(srv, *r): r for r in reqs}

            def finish(t):
                c, m, W, H, flags = by_ticket.pop(t)
                _check_result(ctx, srv, t, clouds[c], m, W, H, flags, oracle)
                pcr.pcr_server_release(srv, t)

            _drain(srv, list(by_ticket), finish)
            assert not by_ticket
            st = pcr.pcr_server_stats_get(srv)
            assert st["completed"] == len(reqs)
            if same_cloud:
                assert st["batches"] < len(reqs)  # views shared batches
            else:
                assert st["batches"] == len(reqs)
        finally:
            pcr.pcr_server_destroy(srv)


def test_shared_stream_cloud_cap_and_completion_queue(ctx, oracle):
    """Three in-flight batches on one stream, at most one cloud per batch;
    finished tickets come out of the completion queue exactly once."""
    clouds = _clouds()
    arena = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    srv = pcr.pcr_server_create(ctx, arena, 160, 120, num_slots=10, max_batch_views=4, max_inflight=3, streams=1,
                                max_batch_clouds=1, background_rgba=BG)
    try:
        for i, c in enumerate(clouds):
            pcr.pcr_server_add_cloud(srv, 20 + i, np.ascontiguousarray(c))
        reqs = _requests(np.random.default_rng(7), clouds, 24, 160, 120)
        by_ticket, pending, seen = {}, list(reqs), []
        t0 = time.time()
        while pending or by_ticket:
            while pending and len(by_ticket) < 10:  # one frame slot per outstanding request
                req = pending.pop(0)
                by_ticket[pcr.pcr_server_submit(srv, 20 + req[0], *req[1:])] = req
            pcr.pcr_server_step(srv)
            for t in pcr.pcr_server_poll_completed(srv, capacity=3):
                assert t not in seen
                seen.append(t)
                c, m, W, H, flags = by_ticket.pop(t)
                _check_result(ctx, srv, t, clouds[c], m, W, H, flags, oracle)
                pcr.pcr_server_release(srv, t)
            assert time.time() - t0 < 60.0, "server did not finish"
        assert len(seen) == len(reqs)
        assert pcr.pcr_server_poll_completed(srv) == []
        st = pcr.pcr_server_stats_get(srv)
        assert st["completed"] == len(reqs) and st["batches"] >= len(clouds)
    finally:
        pcr.pcr_server_destroy(srv)


def test_lru_eviction_keeps_results_exact(ctx, oracle):
    """An arena that holds two of the four clouds: requests cycle through
    them, so clouds are evicted and uploaded again."""
    clouds = [scenes.random_cloud(50_000 + 17 * i, seed=10 + i).numpy() for i in range(4)]
    W, H = 64, 48
    slots = 4
    slot_bytes = 3 * ((8 * W * H + 255) // 256 * 256) + 3 * ((4 * W * H + 255) // 256 * 256)
    ws = (pcr.pcr_batch_workspace_size() + 255) // 256 * 256
    cloud_room = 2 * ((clouds[-1].nbytes + 255) // 256 * 256) + 1024
    arena = torch.empty(slots * slot_bytes + 2 * ws + cloud_room, dtype=torch.uint8, device="cuda")
    srv = pcr.pcr_server_create(ctx, arena, W, H, num_slots=slots, max_batch_views=2, max_inflight=2,
                                background_rgba=BG)
    try:
        host = [np.ascontiguousarray(c) for c in clouds]
        for i, c in enumerate(host):
            pcr.pcr_server_add_cloud(srv, i, c)
        m = scenes.camera((0.2, -2.6, 1.4), (0, 0, 0), (0, 0, 1), W, H)
        order = [0, 1, 2, 3, 0, 2, 1, 3, 3, 0]
        for c in order:
            t = pcr.pcr_server_submit(srv, c, m, W, H, BASIC | HQ)
            _drain(srv, [t])
            _check_result(ctx, srv, t, clouds[c], m, W, H, BASIC | HQ, oracle)
            pcr.pcr_server_release(srv, t)
        st = pcr.pcr_server_stats_get(srv)
        assert st["evictions"] >= 4 and st["uploads"] >= 6
        assert st["resident_clouds"] <= 2
    finally:
        pcr.pcr_server_destroy(srv)


def test_submit_rejections(ctx):
    arena = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    srv = pcr.pcr_server_create(ctx, arena, 32, 32, num_slots=2)
    try:
        cloud = torch.zeros((10, 4), dtype=torch.int32, device="cuda")
        pcr.pcr_server_add_device_cloud(srv, 1, cloud)
        m = np.eye(4, dtype=np.float32)
        for args in [(2, m, 8, 8, BASIC), (1, m, 33, 8, BASIC), (1, m, 8, 8, 0), (1, m, 8, 8, 8)]:
            with pytest.raises(pcr.PcrError) as e:
                pcr.pcr_server_submit(srv, *args)
            assert e.value.status == pcr.PCR_ERR_ARG
        with pytest.raises(pcr.PcrError):
            pcr.pcr_server_add_device_cloud(srv, 1, cloud)  # duplicate id
    finally:
        pcr.pcr_server_destroy(srv)
    with pytest.raises(pcr.PcrError) as e:
        pcr.pcr_server_create(ctx, torch.empty(1 << 20, dtype=torch.uint8, device="cuda"), 1024, 1024, 4)
    assert e.value.status == pcr.PCR_ERR_WORKSPACE
    for kw in [dict(max_inflight=2, streams=3), dict(max_batch_clouds=pcr.PCR_BATCH_MAX_CLOUDS + 1)]:
        with pytest.raises(pcr.PcrError) as e:
            pcr.pcr_server_create(ctx, arena, 32, 32, 2, **kw)
        assert e.value.status == pcr.PCR_ERR_ARG


def test_full_batches_of_small_requests(ctx, oracle):
    """Many small requests, batches of up to 256 views over three clouds; every
    result exact."""
    clouds = [scenes.random_cloud(3001 + 1000 * i, seed=60 + i).numpy() for i in range(3)]
    arena = torch.empty(128 << 20, dtype=torch.uint8, device="cuda")
    srv = pcr.pcr_server_create(ctx, arena, 24, 16, num_slots=300, max_batch_views=pcr.PCR_BATCH_MAX_VIEWS,
                                max_inflight=2, background_rgba=BG)
    try:
        for i, c in enumerate(clouds):
            pcr.pcr_server_add_cloud(srv, i, np.ascontiguousarray(c))
        rng = np.random.default_rng(61)
        reqs = []
        for _ in range(300):
            c = int(rng.integers(0, 3))
            W, H = int(rng.integers(1, 25)), int(rng.integers(1, 17))
            a = rng.uniform(0, 2 * np.pi)
            m = scenes.camera((3 * np.cos(a), 3 * np.sin(a), 1.0), (0, 0, 0), (0, 0, 1), W, H)
            reqs.append((c, m, W, H, int(rng.choice([BASIC, HQ, BASIC | HQ]))))
        tickets = [pcr.pcr_server_submit(srv, *r) for r in reqs]
        _drain(srv, tickets)
        for t, (c, m, W, H, flags) in zip(tickets, reqs):
            _check_result(ctx, srv, t, clouds[c], m, W, H, flags, oracle)
            pcr.pcr_server_release(srv, t)
        st = pcr.pcr_server_stats_get(srv)
        assert st["completed"] == 300 and st["batches"] <= 20
    finally:
        pcr.pcr_server_destroy(srv)


def test_largest_group_policy_keeps_results_exact(ctx, oracle):
    """Largest groups first: batches take the oldest request's cloud and the
    clouds with the most queued requests; every result is still exact, and
    views of one cloud share batches."""
    clouds = _clouds()
    dev = [torch.from_numpy(c.copy()).cuda() for c in clouds]
    arena = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    srv = pcr.pcr_server_create(ctx, arena, 200, 150, num_slots=40, max_batch_views=8, max_inflight=2,
                                max_batch_clouds=2, background_rgba=BG, policy=pcr.PCR_SERVE_LARGEST_GROUP)
    try:
        for i, d in enumerate(dev):
            pcr.pcr_server_add_device_cloud(srv, i, d)
        rng = np.random.default_rng(44)
        reqs = _requests(rng, clouds, 36, 200, 150)
        by_ticket = {pcr.pcr_server_submit(srv, *r): r for r in reqs}

        def finish(t):
            c, m, W, H, flags = by_ticket.pop(t)
            _check_result(ctx, srv, t, clouds[c], m, W, H, flags, oracle)
            pcr.pcr_server_release(srv, t)

        _drain(srv, list(by_ticket), finish)
        assert not by_ticket
        st = pcr.pcr_server_stats_get(srv)
        assert st["completed"] == len(reqs) and st["batches"] <= len(reqs) // 2
    finally:
        pcr.pcr_server_destroy(srv)


def test_admission_bound_and_deadline(ctx, oracle):
    """max_queue refuses submissions beyond it (PCR_ERR_BUSY, nothing queued);
    requests queued past deadline_us expire unrendered and are reported,
    while fresh ones render exactly."""
    cloud = scenes.sphere_plane(30_011, seed=5).numpy()
    dev = torch.from_numpy(cloud.copy()).cuda()
    arena = torch.empty(128 << 20, dtype=torch.uint8, device="cuda")
    W, H = 96, 64
    m = scenes.camera((0, 0, 4), (0, 0, 0), (0, 1, 0), W, H)
    srv = pcr.pcr_server_create(ctx, arena, W, H, num_slots=8, max_batch_views=4, max_inflight=1,
                                background_rgba=BG, max_queue=5, deadline_us=20_000)
    try:
        pcr.pcr_server_add_device_cloud(srv, 0, dev)
        old = [pcr.pcr_server_submit(srv, 0, m, W, H, BASIC) for _ in range(5)]
        with pytest.raises(pcr.PcrError) as e:
            pcr.pcr_server_submit(srv, 0, m, W, H, BASIC)
        assert e.value.status == pcr.PCR_ERR_BUSY
        st = pcr.pcr_server_stats_get(srv)
        assert st["rejected"] == 1 and st["queued"] == 5 and st["submitted"] == 5
        time.sleep(0.05)  # all five are now past their 20 ms deadline
        pcr.pcr_server_step(srv)
        assert [pcr.pcr_server_state(srv, t) for t in old] == [pcr.PCR_REQUEST_EXPIRED] * 5
        assert sorted(pcr.pcr_server_poll_completed(srv)) == sorted(old)
        for t in old:
            res = pcr.pcr_server_get_result(srv, t)
            assert not res.keys and not res.image and res.points == 0 and res.done_us >= res.submit_us
            pcr.pcr_server_release(srv, t)
        st = pcr.pcr_server_stats_get(srv)
        assert st["expired"] == 5 and st["queued"] == 0 and st["batches"] == 0
        fresh = [pcr.pcr_server_submit(srv, 0, m, W, H, f) for f in (BASIC, HQ, BASIC | HQ)]
        _drain(srv, fresh)
        for t, f in zip(fresh, (BASIC, HQ, BASIC | HQ)):
            _check_result(ctx, srv, t, cloud, m, W, H, f, oracle)
            pcr.pcr_server_release(srv, t)
    finally:
        pcr.pcr_server_destroy(srv)
    with pytest.raises(pcr.PcrError) as e:
        pcr.pcr_server_create(ctx, arena, W, H, 2, policy=7)
    assert e.value.status == pcr.PCR_ERR_ARG


def test_l2_budget_changes_passes_not_results(ctx, oracle):
    """The server's L2 budget decides how a batch's views of one cloud are
    packed into passes: at 1 MB every view has a pass of its own (single-view
    kernels), at 1024 MB they all share one.  Results are the same either
    way; a budget above 1024 MB is refused."""
    clouds = _clouds()
    dev = [torch.from_numpy(c.copy()).cuda() for c in clouds]
    arena = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    rng = np.random.default_rng(47)
    reqs = []
    for _ in range(10):
        W, H = int(rng.integers(1, 201)), int(rng.integers(1, 151))
        a = rng.uniform(0, 2 * np.pi)
        m = scenes.camera((3 * np.cos(a), 3 * np.sin(a), 1.5), (0, 0, 0), (0, 0, 1), W, H)
        reqs.append((0, m, W, H, int(rng.choice([BASIC, HQ, BASIC | HQ]))))
    for budget in (1, 1024):
        srv = pcr.pcr_server_create(ctx, arena, 200, 150, num_slots=12, max_batch_views=12, max_inflight=1,
                                    background_rgba=BG, l2_budget_mb=budget)
        try:
            pcr.pcr_server_add_device_cloud(srv, 0, dev[0])
            tickets = {pcr.pcr_server_submit(srv, 0, m, W, H, f): (m, W, H, f) for _, m, W, H, f in reqs}

            def finish(t):
                m, W, H, f = tickets.pop(t)
                _check_result(ctx, srv, t, clouds[0], m, W, H, f, oracle)
                pcr.pcr_server_release(srv, t)

            _drain(srv, list(tickets), finish)
            assert not tickets
        finally:
            pcr.pcr_server_destroy(srv)
    with pytest.raises(pcr.PcrError) as e:
        pcr.pcr_server_create(ctx, arena, 200, 150, 2, l2_budget_mb=1025)
    assert e.value.status == pcr.PCR_ERR_ARG


def test_cancel_queued_requests(ctx, oracle):
    """pcr_server_cancel withdraws a queued request (reported like a finished
    one, with no buffers), refuses one already on the GPU (PCR_ERR_BUSY) and
    unknown or finished tickets (PCR_ERR_ARG); the others render exactly."""
    cloud = scenes.sphere_plane(30_011, seed=6).numpy()
    dev = torch.from_numpy(cloud.copy()).cuda()
    arena = torch.empty(128 << 20, dtype=torch.uint8, device="cuda")
    W, H = 96, 64
    m = scenes.camera((0, 0, 4), (0, 0, 0), (0, 1, 0), W, H)
    srv = pcr.pcr_server_create(ctx, arena, W, H, num_slots=8, max_batch_views=1, max_inflight=1,
                                background_rgba=BG)
    try:
        pcr.pcr_server_add_device_cloud(srv, 0, dev)
        a = pcr.pcr_server_submit(srv, 0, m, W, H, BASIC)
        pcr.pcr_server_step(srv)  # a is launched; b and c wait behind it
        b = pcr.pcr_server_submit(srv, 0, m, W, H, HQ)
        c = pcr.pcr_server_submit(srv, 0, m, W, H, BASIC | HQ)
        assert pcr.pcr_server_state(srv, a) == pcr.PCR_REQUEST_RUNNING
        with pytest.raises(pcr.PcrError) as e:
            pcr.pcr_server_cancel(srv, a)
        assert e.value.status == pcr.PCR_ERR_BUSY
        pcr.pcr_server_cancel(srv, b)
        assert pcr.pcr_server_state(srv, b) == pcr.PCR_REQUEST_CANCELLED
        assert b in pcr.pcr_server_poll_completed(srv)
        res = pcr.pcr_server_get_result(srv, b)
        assert not res.keys and not res.hq_rg and res.points == 0 and res.done_us >= res.submit_us
        with pytest.raises(pcr.PcrError) as e:
            pcr.pcr_server_cancel(srv, b)  # already finished
        assert e.value.status == pcr.PCR_ERR_ARG
        pcr.pcr_server_release(srv, b)
        with pytest.raises(pcr.PcrError) as e:
            pcr.pcr_server_cancel(srv, 10 ** 9)  # unknown ticket
        assert e.value.status == pcr.PCR_ERR_ARG
        _drain(srv, [a, c])
        for t, f in ((a, BASIC), (c, BASIC | HQ)):
            _check_result(ctx, srv, t, cloud, m, W, H, f, oracle)
            pcr.pcr_server_release(srv, t)
        st = pcr.pcr_server_stats_get(srv)
        assert st["cancelled"] == 1 and st["completed"] == 2 and st["queued"] == 0
    finally:
        pcr.pcr_server_destroy(srv)


@pytest.mark.parametrize("seed", range(4))
def test_random_request_streams(ctx, oracle, seed):
    """Seeded random servers (slots, batch size, batches in flight, streams,
    clouds per batch, launch configuration, policy, L2 budget, an arena that
    sometimes holds only some of the clouds) serving random request streams
    over random clouds (special coordinates included) with random cameras,
    sizes and flags, submitted in waves: every result against the oracle."""
    rng = np.random.default_rng(4000 + seed)
    clouds = [random_cloud(rng) for _ in range(int(rng.integers(2, 6)))]
    max_w, max_h = int(rng.integers(8, 160)), int(rng.integers(8, 120))
    slots = int(rng.integers(2, 10))
    inflight = int(rng.integers(1, 4))
    align = lambda b: (b + 255) // 256 * 256  # noqa: E731
    px = max_w * max_h
    slot_bytes = 3 * align(8 * px) + 3 * align(4 * px)
    ws = align(pcr.pcr_batch_workspace_size())
    biggest = max(align(c.nbytes) for c in clouds)
    room = int(rng.integers(2, len(clouds) + 1)) * biggest + 1024
    arena = torch.empty(slots * slot_bytes + inflight * ws + room, dtype=torch.uint8, device="cuda")
    srv = pcr.pcr_server_create(ctx, arena, max_w, max_h, num_slots=slots,
                                max_batch_views=int(rng.integers(1, 9)), max_inflight=inflight,
                                streams=int(rng.integers(1, inflight + 1)),
                                max_batch_clouds=int(rng.integers(0, 3)),
                                batch_config=int(rng.integers(0, pcr.pcr_batch_num_configs())),
                                background_rgba=BG, policy=int(rng.integers(0, 2)),
                                l2_budget_mb=int(rng.choice([0, 1, 64, 1024])))
    try:
        for i, c in enumerate(clouds):
            pcr.pcr_server_add_cloud(srv, 100 + i, np.ascontiguousarray(c))
        by_ticket = {}

        def finish(t):
            c, m, W, H, flags = by_ticket.pop(t)
            _check_result(ctx, srv, t, clouds[c], m, W, H, flags, oracle)
            pcr.pcr_server_release(srv, t)

        tickets = []
        for i in range(int(rng.integers(10, 40))):
            c = int(rng.integers(0, len(clouds)))
            W, H = int(rng.integers(1, max_w + 1)), int(rng.integers(1, max_h + 1))
            flags = int(rng.choice([BASIC, HQ, BASIC | HQ]))
            m = random_matrix(rng, clouds[c], W, H)
            t = pcr.pcr_server_submit(srv, 100 + c, m, W, H, flags)
            by_ticket[t] = (c, m, W, H, flags)
            tickets.append(t)
            if rng.random() < 0.3:
                pcr.pcr_server_step(srv)
        _drain(srv, tickets, finish)
        assert not by_ticket
        assert pcr.pcr_server_stats_get(srv)["completed"] == len(tickets)
    finally:
        pcr.pcr_server_destroy(srv)
