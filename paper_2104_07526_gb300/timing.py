"""Small timing runs through the C ABI, for profiling one part at a time.

    python -m paper_2104_07526_gb300.timing reorder [points] [orders]
        every vertex order (or the comma-separated subset) of the scan scene,
        from its generation order, each once after a warm-up, CUDA events;
    python -m paper_2104_07526_gb300.timing batch
        the 8-cloud x 8-view batch (boxes scenes in shuffled-Morton order,
        basic + HQ), prepared once and launched four times.

Each prints one line of timings.  Run under a profiler, the launches are
the library's own kernels and nothing else of note.
"""
from __future__ import annotations

import json
import sys

ORDERS = {"morton": 0, "morton_shuffle128": 1, "shuffle": 2, "morton63": 3, "morton63_shuffle128": 4}


def time_reorders(n: int, names: list[str]) -> dict:
    import torch
    from . import pcr, scenes
    stream = torch.cuda.current_stream()
    cloud = scenes.scan(n, seed=0, device="cuda")
    ws = torch.empty(pcr.pcr_reorder_workspace_size(n), dtype=torch.uint8, device="cuda")
    out = {}
    with pcr.Context(0, stream=stream) as ctx:
        for name in names:
            best = None
            for _ in range(2):  # the first run warms up
                buf = cloud.clone()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record(stream)
                pcr.pcr_reorder_morton_shuffle128(ctx.handle, buf, n, 0x5EED, ORDERS[name], ws)
                b.record(stream)
                torch.cuda.synchronize()
                t = a.elapsed_time(b)
                best = t if best is None else min(best, t)
                del buf
            out[name] = round(best, 3)
    return out


def time_batch(launches: int = 4) -> dict:
    import torch
    from . import pcr, scenes
    stream = torch.cuda.current_stream()
    clouds = [scenes.boxes(nc, seed=i, device="cuda") for i, nc in enumerate(scenes.BATCH_CLOUD_SIZES)]
    views = scenes.batch_views(len(clouds))
    bufs = []
    for _, v in views:
        npx = v.width * v.height
        bufs.append({k: torch.empty(npx, dtype=t, device="cuda") for k, t in
                     (("keys", torch.int64), ("image", torch.int32), ("hq_depth", torch.int32),
                      ("hq_rg", torch.int64), ("hq_ba", torch.int64), ("hq_image", torch.int32))})
    flags = pcr.PCR_BATCH_BASIC | pcr.PCR_BATCH_HQ
    with pcr.Context(0, stream=stream) as ctx:
        h = ctx.handle
        # shuffled-Morton order first, as the benchmark's batched workload
        rws = torch.empty(pcr.pcr_reorder_workspace_size(max(c.shape[0] for c in clouds)), dtype=torch.uint8,
                          device="cuda")
        for c in clouds:
            pcr.pcr_reorder_morton_shuffle128(h, c, c.shape[0], 0x5EED, pcr.PCR_ORDER_MORTON_SHUFFLE128, rws)
        torch.cuda.synchronize()
        del rws
        torch.cuda.empty_cache()
        ws = torch.empty(pcr.pcr_batch_workspace_size(), dtype=torch.uint8, device="cuda")
        pcr.pcr_batch_prepare(h, [pcr.batch_cloud(c) for c in clouds],
                              [pcr.batch_view(v.matrix, v.width, v.height, c, flags, **b) for (c, v), b in
                               zip(views, bufs)], 1.01, 0, ws)
        times = []
        for _ in range(launches):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pcr.pcr_batch_launch(h, ws, 0)
            b.record(stream)
            torch.cuda.synchronize()
            times.append(round(a.elapsed_time(b), 3))
    return {"batch_ms": times}


def main(argv: list[str]) -> int:
    from . import build
    build.build()
    if not argv or argv[0] not in ("reorder", "batch"):
        print(__doc__)
        return 2
    if argv[0] == "reorder":
        n = int(argv[1]) if len(argv) > 1 else 100_000_000
        names = argv[2].split(",") if len(argv) > 2 else list(ORDERS)
        print(json.dumps(time_reorders(n, names)), flush=True)
    else:
        print(json.dumps(time_batch()), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
