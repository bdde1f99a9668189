"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

bench.py runs one replica per GPU (the path needs no data exchange); the
only cross-rank steps are a barrier and the maximum of the timed region.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

from conftest import ROOT


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench
    r, w, local = bench.dist_env()
    dist = bench.dist_init(w, "gloo")
    bench.barrier(dist)
    slowest = bench.max_over_ranks(1.5 + rank, dist)
    value = bench.aggregate_throughput(1000, w, slowest)
    out.put((r, w, local, slowest, value))
    dist.destroy_process_group()


def test_two_ranks_max_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in results] == [(0, 2, 0), (1, 2, 1)]
    # every rank sees the slowest rank's time; throughput counts both ranks' points
    assert all(r[3] == 2.5 for r in results)
    assert all(r[4] == pytest.approx(2000 / 2.5) for r in results)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_init(1, "gloo") is None
    assert bench.max_over_ranks(3.0, None) == 3.0
    assert bench.aggregate_throughput(800, 1, 2.0) == 400.0
