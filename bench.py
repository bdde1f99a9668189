#!/usr/bin/env python3
"""Benchmark of compute-based point rendering on GB300.

Workload (default): the 800M-point scan-like scene (facade walls plus a
terrain heightfield, 12.8 GB of 16-byte records), reordered once to shuffled
Morton order (batches of 128), rendered at 1920x1080 from the overview
camera.  One step is one basic frame: clear the key buffer, render with warp
deduplication plus early depth test (the paper's "dedup" method), resolve to
rgba.  The metric is points per second; the dominant kernel (the render pass)
is also reported as achieved HBM GB/s against the measured copy bandwidth.

The same JSON line carries the end-to-end number (points uploaded from pinned
host memory through pcr_upload_points_from_host, frame, image read back
through pcr_download, every step), per-phase times, the one-time reorder
cost, a sweep over render variants, vertex orders and cameras, and the CPU
oracle timed on a bounded sample of the same frame.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --impl reference the CPU oracle is timed instead (rank 0 only).  Under
torchrun each rank renders its own copy of the workload on its own GPU (weak
scaling, replicas only: no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "points/s and HBM GB/s vs roofline per frame"
UNIT = "points/s"
POINT_BYTES = 16
FALLBACK_HBM_GBS = 6800.0
# Nominal HBM3e bandwidth of a GB300 ("about 8 TB/s"), reported beside the
# measured copy bandwidth.
NOMINAL_HBM_GBS = 8000.0
# The timed frame's variant.  Every exact variant leaves the same buffer; on
# the scan scene's overview in shuffled-Morton order, early-z with warp
# deduplication (Sec. 3.4, the paper's fastest) is 1-2% faster than the early
# test alone, and the two lead the rest (the sweep in the JSON line times all
# of them).
HEADLINE_VARIANT = "dedup+early-z"
# The HQ frames' depth-pass variant (the colour pass sums colours inside the
# warp for every variant but atomicMin): with the early test the depth pass
# is the same for early-z and dedup+early-z up to the deduplication, which
# is about 1.5% faster on the scan scene's HQ frames.
HQ_VARIANT = "dedup+early-z"

CONFIGS = {
    # name: (points, generator, views, headline view)
    "scan800M": dict(points=800_000_000, gen="scan", view="overview",
                     desc="800M-point scan scene (facades + terrain), shuffled-Morton order, overview camera, "
                          f"1920x1080, basic frame with {HEADLINE_VARIANT}"),
    "scan100M": dict(points=100_000_000, gen="scan", view="overview",
                     desc="100M-point scan scene (the 800M recipe at 1/8 size, for profiling), shuffled-Morton "
                          "order, overview camera, 1920x1080, basic frame"),
    "boxes50M": dict(points=50_000_000, gen="boxes", view="overview",
                     desc="50M points on 200 boxes over a ground plane, shuffled-Morton order, overview camera, "
                          f"1920x1080, basic frame with {HEADLINE_VARIANT}"),
    "sphere1M": dict(points=1_000_000, gen="sphere_plane", view="front",
                     desc="1M points on a sphere plus a plane, shuffled-Morton order, 640x480, basic frame with "
                          f"{HEADLINE_VARIANT}"),
}


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=sorted(CONFIGS), default="scan800M")
    ap.add_argument("--no-sweep", action="store_true", help="skip the variant x order x camera sweep")
    ap.add_argument("--no-small", action="store_true", help="skip the 1M and 50M-point workloads")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffers) measurement")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--variant", default=HEADLINE_VARIANT, help="render variant of the timed frame")
    ap.add_argument("--order", choices=["morton_shuffle128", "morton", "shuffle", "original"],
                    default="morton_shuffle128", help="vertex order of the timed frame (profiling)")
    ap.add_argument("--no-hq", action="store_true", help="skip the high-quality frame")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched (8 clouds x 8 views) measurement")
    ap.add_argument("--no-served", action="store_true", help="skip the served (Poisson request stream) measurement")
    ap.add_argument("--served-seconds", type=float, default=2.0, help="length of the served request stream")
    ap.add_argument("--part", choices=["reorder", "batch", "served"],
                    help="time one part alone and print its timings (for running under a profiler): every "
                         "vertex order of the scan scene (--points, --orders), the 8-cloud x 8-view batch, or "
                         "the saturated request stream through the server alone (--served-seconds)")
    ap.add_argument("--points", type=int, default=100_000_000, help="scan-scene points for --part reorder")
    ap.add_argument("--orders", default="morton,morton_shuffle128,shuffle,morton63,morton63_shuffle128",
                    help="comma-separated vertex orders for --part reorder")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------

def sections(args, world: int) -> dict:
    """Which parts of the run take place.  The timed frame always runs; the
    HQ frames and e2e follow their flags at any N.  The characterisations of
    one GPU (the variant sweep and 63-bit reorders, the smaller workloads,
    the batched and served workloads) and the CPU baseline run at N = 1 only:
    under torchrun every rank would repeat them on its own GPU, and the
    served workload alone holds about 18 GB of host memory per rank."""
    single = world == 1
    return {"hq": not args.no_hq, "e2e": not args.no_e2e, "sweep": single and not args.no_sweep,
            "batched": single and not args.no_batched, "small": single and not args.no_small,
            "served": single and not args.no_served, "cpu": single and not args.no_cpu}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world: int, backend: str):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return dist if world > 1 else None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(value: float, dist, device=None) -> float:
    """Largest value over all ranks (timing only; not on the data path)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(points_per_rank: int, world: int, max_seconds: float) -> float:
    """Whole-job points/s: every rank's points over the slowest rank's time."""
    return points_per_rank * world / max_seconds


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_id: str, interval_ms: int = 50):
        self.gpu_id = gpu_id
        self.interval_ms = interval_ms
        self.proc = None
        self.lines: list[tuple[float, str]] = []
        self.reader = None
        self.window = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.interval_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, start: float, end: float):
        """Keep only samples that arrived inside [start, end] (host clock)."""
        self.window = (start, end)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.reader.join(timeout=5)
        sm, smax, power, reasons = [], [], [], set()
        for t, line in self.lines:
            if self.window is not None and not (self.window[0] <= t <= self.window[1]):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, state in zip(self.REASONS, parts[5:9]):
                if state.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


def nvsmi_id(cuda_index: int) -> str:
    """nvidia-smi id of a CUDA device (its UUID; CUDA_VISIBLE_DEVICES may
    renumber devices)."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(cuda_index).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(cuda_index)


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def measured_hbm_gbs() -> tuple[float, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


TRAFFIC_RECORD = "traffic_render_scan100M.txt"


def recorded_traffic(kernel_sources: list[str], variant: str, points: int) -> dict | None:
    """DRAM bytes per render launch from an ncu capture of a smaller case of
    the same scene (profiles/traffic_render_scan100M.txt), scaled to the
    launch's points: the render streams every point once, so its traffic
    grows with the point count.  Reported only while the capture was taken on
    the current kernel sources and the timed variant."""
    path = os.path.join(ROOT, "profiles", TRAFFIC_RECORD)
    try:
        with open(path) as f:
            kv = dict(line.split("=", 1) for line in f.read().splitlines() if "=" in line and not line.startswith("#"))
    except OSError:
        return None
    h = hashlib.sha256()
    for p in kernel_sources:
        with open(p, "rb") as f:
            h.update(f.read())
    if kv.get("sources_sha256", "").strip() != h.hexdigest() or kv.get("variant", "").strip() != variant:
        return None
    captured = int(kv["points"])
    per_point = float(kv["bytes_per_launch"]) / captured
    return {"bytes_per_launch": per_point * points, "captured_points": captured,
            "captured_bytes_per_launch": float(kv["bytes_per_launch"]), "note": kv.get("note", "").strip()}


def make_cloud(cfg: dict, device, seed: int = 0):
    from paper_2104_07526_gb300 import scenes
    n = cfg["points"]
    if cfg["gen"] == "scan":
        cloud = scenes.scan(n, seed=seed, device=device)
        views = scenes.scan_views(n, seed)
    elif cfg["gen"] == "boxes":
        cloud = scenes.boxes(n, seed=seed, device=device)
        views = scenes.boxes_views(seed)
    else:
        cloud = scenes.sphere_plane(n, seed=seed, device=device)
        views = scenes.sphere_plane_views()
    return cloud, views


def cpu_sample_indices(n: int, sample: int):
    import torch
    stride = max(1, n // max(sample, 1))
    return torch.arange(0, n, stride, dtype=torch.int64)[:sample]


def describe_sample(n: int, sample: int) -> str:
    stride = max(1, n // max(sample, 1))
    if stride == 1:
        return f"the first {sample} of the {n} points"
    return f"every {stride}th point of the {n}-point cloud ({sample} points)"


def time_oracle(pts_np: np.ndarray, view, repeats: int = 1, threads: int = 1) -> float:
    """Seconds per oracle frame (render + resolve) on this sample: the
    single-threaded functions for threads == 1, else their host-parallel
    forms on `threads` threads (0 = every host core)."""
    from oracle import pyoracle
    best = None
    for _ in range(repeats):
        t0 = time.perf_counter()
        if threads == 1:
            keys = pyoracle.render_basic(pts_np, view.matrix, view.width, view.height)
            pyoracle.resolve_basic(keys, pts_np, 0)
        else:
            keys, _ = pyoracle.render_basic_threads(pts_np, view.matrix, view.width, view.height, threads)
            pyoracle.resolve_basic_threads(keys, pts_np, 0, threads)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return best


# Algorithmic DRAM bytes per point of each one-time reorder (Sec. 4, Sec. 5):
# what any sort-based reorder must move at least once, counted as 16 B of
# records read for the bounds, 16 B read for the codes, every radix pass
# reading and writing a 4-byte key and a 4-byte value (16 B), and the final
# record gather (16 B read, 16 B written).  The shuffle's keys come from the
# point index: 8 B written instead of the two record reads.  Morton codes of
# 30 bits and the 32-bit shuffle keys sort in 4 passes; 63-bit codes in 8.
REORDER_ALGORITHMIC_BYTES_PER_POINT = {
    "morton": 16 + 16 + 4 * 16 + 32,
    "morton_shuffle128": 16 + 16 + 4 * 16 + 32,
    "shuffle": 8 + 4 * 16 + 32,
    "morton63": 16 + 16 + 8 * 16 + 32,
    "morton63_shuffle128": 16 + 16 + 8 * 16 + 32,
}

# DRAM bytes per point this design moves (its own choices included):
#   bounds 16 read (plus 16 written: the record copy, for the 30-bit orders);
#   30-bit codes 16 read + 4 written (the key); 63-bit codes 16 read + 8
#   written (low key, high word); each sort pass 4 (histogram read) + 8 read
#   + 8 written (key, index), less the 4 + 4 the first pass does not read (the
#   kernel that made the keys counted its digits, and it makes the indices),
#   and 4 + 4 more for the high word the 63-bit orders carry through their
#   first sort (whose last pass writes no keys).  The last pass of the sort
#   that orders the records writes no key and no index: it moves each record
#   from the copy to its final position (16 read, 16 written).  Batch sort and
#   batch slots about 1; separate record copy (63-bit orders) 16 + 16.  The
#   shuffle writes its 4-byte random keys, then each of its four passes reads
#   4 (histogram; not the first) and moves the key and the 16-byte record it
#   carries (20 read, 20 written; the last writes no key).
REORDER_BYTES_PER_POINT = {
    "morton": 32 + 20 + 4 * 20 - 8 - 8 + 32,
    "morton_shuffle128": 32 + 20 + 4 * 20 - 8 - 8 + 32 + 1,
    "shuffle": 4 + 4 * (4 + 40) - 4 - 4,
    "morton63": 16 + 24 + 4 * 28 - 8 - 4 + 32 + 4 * 20 - 8 + 32,
    "morton63_shuffle128": 16 + 24 + 4 * 28 - 8 - 4 + 32 + 4 * 20 - 8 + 32 + 1,
}


def reorder_roofline(reorder_ms: dict, n: int, peak: float) -> dict:
    """Per order: the algorithmic bytes over the time as a fraction of the
    peak, and this design's own bytes as a ratio to the algorithmic ones."""
    out = {}
    for name, ms in reorder_ms.items():
        gb = REORDER_ALGORITHMIC_BYTES_PER_POINT[name] * n / 1e9
        design_gb = REORDER_BYTES_PER_POINT[name] * n / 1e9
        out[name] = {"ms": ms, "algorithmic_gb": gb, "achieved_gbs": gb / (ms * 1e-3), "frac": gb / (ms * 1e-3) / peak,
                     "design_gb": design_gb, "design_over_algorithmic": design_gb / gb,
                     "design_gbs": design_gb / (ms * 1e-3)}
    return out


def oracle_threads() -> int:
    """Host threads the parallel oracle uses."""
    from oracle import pyoracle
    _, used = pyoracle.render_basic_threads(np.zeros((0, 4), np.int32), np.eye(4, dtype=np.float32), 1, 1, 0)
    return used


def oracle_baseline(cloud_host_fn, n: int, view, target_s: float) -> dict:
    """Time the CPU oracle as it stands on the host cores: its host-parallel
    render and resolve on every core, on a sample of the same cloud sized to
    about target_s seconds of work, plus the single-threaded functions on
    the same sample for about a third of that."""

    def timed(threads: int, seconds: float):
        pilot_n = min(n, 4_000_000)
        pilot = cloud_host_fn(pilot_n)
        t = time_oracle(pilot, view, repeats=2, threads=threads)  # the first pass pays for page faults
        rate = pilot_n / max(t, 1e-6)
        sample = int(min(n, max(pilot_n, rate * seconds)))
        pts = cloud_host_fn(sample)
        # whole frames until the time is spent (the sample is capped at the
        # cloud, which a fast host renders in less than the target)
        frames, total = 0, 0.0
        while total < seconds and frames < 10:
            total += time_oracle(pts, view, threads=threads)
            frames += 1
        return sample * frames / total, sample, frames, total

    cores = oracle_threads()
    value, sample, frames, total = timed(0, target_s)
    one, one_sample, one_frames, one_total = timed(1, target_s / 3)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{describe_sample(n, sample)}, {frames} frame(s) (render + resolve), C oracle on "
                      f"{cores} threads, {total:.2f} s",
            "single_thread": {"value": one, "unit": UNIT, "cores": 1,
                              "sample": f"{describe_sample(n, one_sample)}, {one_frames} frame(s), {one_total:.2f} s"}}


def run_small_configs(h, pcr, stream, dev, with_cpu: bool) -> dict:
    """The two smaller workloads beside the headline one, each as its
    configuration states it, in generation order: the 1M-point sphere-and-
    plane scene (640x480, L2-resident points), basic atomicMin frame; the
    50M-point boxes scene, every camera (overview, mid, inside a box) with
    the basic, dedup, early-z and HQ frames.  Beside them, the same frames
    after the paper's recommended shuffled-Morton reorder.  A basic frame is
    clear + render + resolve, an HQ frame clear + depth + colours + resolve,
    timed with CUDA events.  CPU baselines: the oracle's host-parallel and
    single-threaded basic frames on the whole cloud."""
    import torch
    basic = {"atomicMin": pcr.PCR_VARIANT_ATOMICMIN, "dedup": pcr.PCR_VARIANT_DEDUP,
             "early-z": pcr.PCR_VARIANT_EARLYZ, "dedup+early-z": pcr.PCR_VARIANT_DEDUP_EARLYZ}
    plan = {"sphere1M": (["atomicMin", "early-z"], False), "boxes50M": (list(basic), True)}
    out = {}
    for name in ("sphere1M", "boxes50M"):
        cfg = CONFIGS[name]
        variants, with_hq = plan[name]
        cloud, views = make_cloud(cfg, dev)
        n = cloud.shape[0]
        reps = 200 if n <= 10_000_000 else 50
        W, H = max(v.width for v in views), max(v.height for v in views)
        fb = pcr.alloc_framebuffer(W, H, dev)
        pcr.pcr_set_framebuffer(h, fb["keys"], fb["hq_depth"], fb["hq_rg"], fb["hq_ba"])

        def frames(graphs: dict | None = None):
            pcr.pcr_upload_points(h, cloud, n)
            res = {}
            for v in views:
                pcr.pcr_set_matrix(h, v.matrix)
                pcr.pcr_set_viewport(h, v.width, v.height)
                row = {}
                for vname in variants:
                    def frame(var=basic[vname]):
                        pcr.pcr_clear(h, pcr.PCR_CLEAR_KEYS)
                        pcr.pcr_render_basic(h, var, False)
                        pcr.pcr_resolve(h, pcr.PCR_RESOLVE_BASIC, fb["image"], 0)
                    row[vname] = round(time_loop(frame, stream, reps=reps, warm=5), 4)
                    if graphs is not None:
                        # the same frame recorded once and replayed as one graph launch
                        pcr.pcr_capture_begin(h)
                        frame()
                        g = pcr.pcr_capture_end(h)
                        graphs.setdefault(v.name, {})[vname] = round(
                            time_loop(lambda: pcr.pcr_graph_launch(h, g), stream, reps=reps, warm=5), 4)
                        pcr.pcr_graph_destroy(g)
                if with_hq:
                    def hq_frame():
                        pcr.pcr_render_hq(h, 1.01, pcr.PCR_VARIANT_DEDUP_EARLYZ, True)
                        pcr.pcr_resolve(h, pcr.PCR_RESOLVE_HQ, fb["image"], 0)
                    row["hq"] = round(time_loop(hq_frame, stream, reps=reps, warm=5), 4)
                res[v.name] = row
            return res

        launch_bound = n <= 10_000_000  # small clouds: launches, not the point stream, set the frame time
        g_orig, g_reord = ({}, {}) if launch_bound else (None, None)
        original = frames(g_orig)
        vertex_order(h, pcr, [cloud], dev)
        reordered = frames(g_reord)
        head = next(v for v in views if v.name == cfg["view"])
        first = variants[0]
        ms = original[head.name][first]
        row = {"points": n, "width": head.width, "height": head.height, "camera": head.name,
               "order": "original", "variant": first, "gpu_frame_ms": ms, "gpu_points_per_s": n / (ms * 1e-3),
               "frames": reps, "frame_ms": {"original": original, "morton_shuffle128": reordered}}
        if launch_bound:
            row["graph_frame_ms"] = {"original": g_orig, "morton_shuffle128": g_reord}
        if with_cpu:
            host = cloud.cpu().numpy()
            t_all = time_oracle(host, head, repeats=2, threads=0)
            t_one = time_oracle(host, head, repeats=1, threads=1)
            row["cpu_baseline"] = {"kind": "oracle", "cores": oracle_threads(), "frame_ms": t_all * 1e3,
                                   "points_per_s": n / t_all, "single_thread_frame_ms": t_one * 1e3,
                                   "single_thread_points_per_s": n / t_one,
                                   "sample": "the whole cloud, best of 2 frames (1 single-threaded)"}
        out[name] = row
        del cloud, fb
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------

def run_reference(args, cfg):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import torch
    from paper_2104_07526_gb300 import scenes
    from oracle import build as oracle_build
    oracle_build.build()
    n = cfg["points"]
    _, views = make_cloud({**cfg, "points": 1024}, "cpu") if cfg["gen"] != "scan" else (None, scenes.scan_views(n, 0))
    view = next(v for v in views if v.name == cfg["view"])

    from oracle import pyoracle

    def host_sample(k):
        """A strided sample of the generated cloud, put in shuffled-Morton
        order by the oracle (untimed), as the timed workload is."""
        idx = cpu_sample_indices(n, k)
        if cfg["gen"] == "scan":
            pts = scenes.scan(n, seed=0, indices=idx).numpy()
        else:
            full, _ = make_cloud(cfg, "cpu")
            pts = full[idx].numpy()
        return pyoracle.gather(pts, pyoracle.reorder(pts, 0x5EED, pyoracle.MORTON_SHUFFLE))

    # size each step so warmup + steps stay within about two minutes
    budget = 120.0
    pilot_n = min(n, 1_000_000)
    pilot = host_sample(pilot_n)
    rate = pilot_n / max(time_oracle(pilot, view, threads=0), 1e-6)
    per_step = budget / max(1, args.steps + args.warmup)
    # at most 100M points: the oracle puts the sample in shuffled-Morton order
    # (a single-threaded sort) before timing, which must stay a few minutes
    sample = int(min(n, 100_000_000, max(100_000, rate * per_step)))
    pts = host_sample(sample)
    for _ in range(args.warmup):
        time_oracle(pts, view, threads=0)
    times = [time_oracle(pts, view, threads=0) for _ in range(args.steps)]
    step_s = sum(times) / len(times)
    value = sample / step_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32/u64", "data": "synthetic",
        "config": {**workload_config(cfg, view, args.variant), "sample_points": sample,
                   "sample": f"timed on {describe_sample(n, sample)}, in shuffled-Morton order"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                         "sample": f"per step {describe_sample(n, sample)}, put in shuffled-Morton order, "
                                   f"render + resolve, C oracle on every host core"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


ORDER_WORDS = {"morton_shuffle128": "shuffled-Morton order", "morton": "Morton order", "shuffle": "shuffled order",
               "original": "original (generation) order"}


def workload_config(cfg: dict, view, variant: str, order: str = "morton_shuffle128") -> dict:
    desc = cfg["desc"].replace(f"basic frame with {HEADLINE_VARIANT}", f"basic frame with {variant}")
    desc = desc.replace("shuffled-Morton order", ORDER_WORDS[order])
    return {"workload": desc, "points": cfg["points"], "width": view.width, "height": view.height,
            "order": order, "camera": view.name, "variant": variant,
            "l2": "inputs larger than L2 (no flush needed)" if cfg["points"] * POINT_BYTES > 129e6
            else "inputs fit in L2 (L2-resident case)", "parallelism": "replicas"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, cfg):
    import torch
    from paper_2104_07526_gb300 import build as lib_build
    from paper_2104_07526_gb300 import pcr

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    lib_build.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    n = cfg["points"]

    t0 = time.perf_counter()
    cloud, views = make_cloud(cfg, dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    view = next(v for v in views if v.name == cfg["view"])
    W, H = view.width, view.height

    ctx = pcr.Context(local, stream=stream)
    h = ctx.handle
    fb = pcr.alloc_framebuffer(W, H, dev)
    pcr.pcr_set_framebuffer(h, fb["keys"], fb["hq_depth"], fb["hq_rg"], fb["hq_ba"])
    pcr.pcr_set_lock_buffer(h, fb["locks"], 0)

    # --- one-time reorders (Sec. 4); original order kept for the sweep ----
    ws = torch.empty(pcr.pcr_reorder_workspace_size(n), dtype=torch.uint8, device=dev)
    orders = {"original": cloud}
    reorder_ms = {}
    for name, mode in (("morton", pcr.PCR_ORDER_MORTON), ("shuffle", pcr.PCR_ORDER_SHUFFLE),
                       ("morton_shuffle128", pcr.PCR_ORDER_MORTON_SHUFFLE128)):
        if args.no_sweep and name not in ("morton_shuffle128", args.order):
            continue
        buf = cloud.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pcr.pcr_reorder_morton_shuffle128(h, buf, n, 0x5EED, mode, ws)
        e1.record(stream)
        torch.cuda.synchronize()
        reorder_ms[name] = e0.elapsed_time(e1)
        orders[name] = buf
    run = sections(args, world)
    if run["sweep"]:
        # the paper's 21-level Morton code (63 bits): timed, not kept
        for name, mode in (("morton63", pcr.PCR_ORDER_MORTON63),
                           ("morton63_shuffle128", pcr.PCR_ORDER_MORTON63_SHUFFLE128)):
            buf = cloud.clone()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pcr.pcr_reorder_morton_shuffle128(h, buf, n, 0x5EED, mode, ws)
            e1.record(stream)
            torch.cuda.synchronize()
            reorder_ms[name] = e0.elapsed_time(e1)
            del buf
    del ws
    points = orders[args.order]
    if args.no_sweep:
        for name in [k for k in orders if k != args.order]:
            del orders[name]
        del cloud
    torch.cuda.empty_cache()

    def set_view(v):
        pcr.pcr_set_matrix(h, v.matrix)
        pcr.pcr_set_viewport(h, v.width, v.height)

    names = {v: k for k, v in pcr.VARIANT_NAMES.items()}
    variant = names[args.variant]
    pcr.pcr_upload_points(h, points, n)
    set_view(view)

    def frame():
        pcr.pcr_clear(h, pcr.PCR_CLEAR_KEYS)
        pcr.pcr_render_basic(h, variant, False)
        pcr.pcr_resolve(h, pcr.PCR_RESOLVE_BASIC, fb["image"], 0)

    # --- timed region ---------------------------------------------------------
    for _ in range(args.warmup):
        frame()
    clocks = ClockSampler(nvsmi_id(local))
    clocks.start()
    time.sleep(0.5)  # nvidia-smi start-up
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    torch.cuda.synchronize()
    barrier(dist)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_begin = time.time()
    start.record(stream)
    for k in range(K):
        ev[k][0].record(stream)
        pcr.pcr_clear(h, pcr.PCR_CLEAR_KEYS)
        ev[k][1].record(stream)
        pcr.pcr_render_basic(h, variant, False)
        ev[k][2].record(stream)
        pcr.pcr_resolve(h, pcr.PCR_RESOLVE_BASIC, fb["image"], 0)
        ev[k][3].record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    t_end = time.time()
    barrier(dist)
    torch.cuda.synchronize()
    clocks.mark(t_begin, t_end)
    clock_info = clocks.stop()
    total_ms = start.elapsed_time(end)
    max_total_ms = max_over_ranks(total_ms, dist, dev)
    ms_per_step = max_total_ms / K
    phase = {p: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in ev) for i, p in
             enumerate(("clear", "render", "resolve"))}
    frame_times = [e[0].elapsed_time(e[3]) for e in ev]
    render_times = [e[1].elapsed_time(e[2]) for e in ev]
    frame_stats = {"frame_ms_median": statistics.median(frame_times), "frame_ms_min": min(frame_times),
                   "frame_ms_max": max(frame_times), "render_ms_median": statistics.median(render_times)}
    render_ms = phase["render"]
    value = aggregate_throughput(n, world, max_total_ms / K / 1e3)

    peak, peak_src = measured_hbm_gbs()
    achieved = n * POINT_BYTES / (render_ms * 1e-3) / 1e9
    traffic = recorded_traffic([os.path.join(ROOT, "paper_2104_07526_gb300", "csrc", f)
                                for f in ("render.cu", "common.cuh", "geometry.cuh")], args.variant, n) \
        if cfg["gen"] == "scan" else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "nominal_peak": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS,
                "traffic": traffic["bytes_per_launch"] if traffic else None,
                "traffic_source": (f"ncu DRAM bytes of a {traffic['captured_points'] // 1_000_000}M-point launch of "
                                   f"the same scene, scaled to {n // 1_000_000}M points") if traffic else None,
                "kernel": f"k_render_basic<{args.variant}>", "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"
                if peak_src == "measured" else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": n * POINT_BYTES}

    # --- HQ frame (Sec. 3.5) ------------------------------------------------------
    hq_variant = names[HQ_VARIANT]

    def hq_frame():
        pcr.pcr_render_hq(h, 1.01, hq_variant, True)
        pcr.pcr_resolve(h, pcr.PCR_RESOLVE_HQ, fb["image"], 0)

    def hq1r_frame():
        pcr.pcr_render_hq1r(h, 1.01, hq_variant, True)
        pcr.pcr_resolve(h, pcr.PCR_RESOLVE_HQ1R, fb["image"], 0)

    pcr.pcr_set_hq1r_buffer(h, fb["hq1r_primary"])
    hq_ms = time_loop(hq_frame, stream, reps=max(5, min(K, 50)), warm=3) if run["hq"] else None
    hq1r_ms = time_loop(hq1r_frame, stream, reps=max(5, min(K, 50)), warm=3) if run["hq"] else None

    # --- end to end through the C ABI with host buffers ---------------------------
    e2e = None
    if run["e2e"]:
        e2e = run_e2e(h, pcr, points, n, fb, W, H, variant, stream, dist, dev, world,
                      steps=max(3, min(K, 20)), warm=2)
        pcr.pcr_upload_points(h, points, n)

    # --- sweep: variants x orders x cameras ---------------------------------------
    sweep = None
    if run["sweep"]:
        sweep = run_sweep(h, pcr, orders, views, n, fb, stream)
        pcr.pcr_upload_points(h, points, n)
        set_view(view)

    # --- batched: 8 clouds x 8 views, per-view calls vs one graph -----------------
    batched = None
    if run["batched"]:
        batched = run_batched(h, pcr, stream, dev, reps=max(3, min(K, 10)))
        pcr.pcr_upload_points(h, points, n)
        set_view(view)
        pcr.pcr_set_framebuffer(h, fb["keys"], fb["hq_depth"], fb["hq_rg"], fb["hq_ba"])

    # --- CPU oracle baseline (rank 0, one GPU) -------------------------------------
    cpu = None
    if rank == 0 and run["cpu"]:
        from oracle import build as oracle_build
        oracle_build.build()
        cpu = oracle_baseline(lambda k: points[cpu_sample_indices(n, k).to(dev)].cpu().numpy(), n, view,
                              args.cpu_seconds)

    # --- the smaller workloads (1M and 50M points), GPU frame and CPU oracle --
    small = None
    if run["small"]:
        small = run_small_configs(h, pcr, stream, dev, with_cpu=(rank == 0 and run["cpu"]))
        pcr.pcr_upload_points(h, points, n)
        set_view(view)
        pcr.pcr_set_framebuffer(h, fb["keys"], fb["hq_depth"], fb["hq_rg"], fb["hq_ba"])

    # --- served: Poisson request stream, continuous batching vs plain launches --
    served = served_sat = None
    if run["served"]:
        orders.clear()
        points = cloud = None
        torch.cuda.empty_cache()
        served, served_sat = run_served(h, pcr, stream, dev, args.served_seconds, rates=(2000.0, 8000.0))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/u64", "data": "synthetic", "config": workload_config(cfg, view, args.variant, args.order),
            "frame_gbs": n * POINT_BYTES / (ms_per_step * 1e-3) / 1e9,
            "phases_ms": phase, "frame_stats": frame_stats, "hq_frame_ms": hq_ms, "hq1r_frame_ms": hq1r_ms,
            "hq_roofline": None if hq_ms is None else {
                "bound": "hbm", "algorithmic_bytes": 2 * n * POINT_BYTES,
                "achieved_gbs": 2 * n * POINT_BYTES / (hq_ms * 1e-3) / 1e9,
                "frac": 2 * n * POINT_BYTES / (hq_ms * 1e-3) / 1e9 / peak,
                "frac_nominal": 2 * n * POINT_BYTES / (hq_ms * 1e-3) / 1e9 / NOMINAL_HBM_GBS,
                "note": "two passes over the points"},
            "reorder_roofline": reorder_roofline(reorder_ms, n, peak),
            "roofline": roofline, "clocks": clock_info, "gpu_launches": 3 * K,
            "e2e": e2e, "cpu_baseline": cpu, "reorder_ms": reorder_ms, "generate_s": gen_s,
            "sweep_ms": sweep, "small_configs": small, "batched": batched, "served": served,
            "served_saturated": served_sat,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def time_loop(fn, stream, reps: int, warm: int) -> float:
    import torch
    for _ in range(warm):
        fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def run_e2e(h, pcr, points, n, fb, W, H, variant, stream, dist, dev, world, steps: int, warm: int) -> dict:
    """Points from pinned host memory -> frame -> image back to host, every
    step, all through the C ABI.  Two ways in: the render kernels read the
    pinned buffer over the host link (pcr_upload_points_mapped, the reported
    value), or the library copies it into a device buffer first
    (pcr_upload_points_from_host, reported as `copy_path`).  Both move every
    point record host -> device once per step."""
    import torch
    host = torch.empty(points.shape, dtype=points.dtype, pin_memory=True)
    host.copy_(points)
    img_host = torch.empty(W * H, dtype=torch.int32).pin_memory()

    def frame_and_download():
        pcr.pcr_clear(h, pcr.PCR_CLEAR_KEYS)
        pcr.pcr_render_basic(h, variant, False)
        pcr.pcr_resolve(h, pcr.PCR_RESOLVE_BASIC, fb["image"], 0)
        pcr.pcr_download(h, img_host, fb["image"])  # synchronous

    def step_mapped():
        pcr.pcr_upload_points_mapped(h, host, n)
        frame_and_download()

    def step_copy():
        pcr.pcr_upload_points_from_host(h, points, host, n)
        frame_and_download()

    def measure(step) -> dict:
        for _ in range(warm):
            step()
        torch.cuda.synchronize()
        barrier(dist)
        t0 = time.perf_counter()
        marks = []
        for _ in range(steps):
            step()
            marks.append(time.perf_counter())
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, dist, dev)
        per = [(b - a) * 1e3 for a, b in zip([t0] + marks[:-1], marks)]
        return {"value": aggregate_throughput(n, world, dt / steps), "unit": UNIT,
                "h2d_bytes_per_step": n * POINT_BYTES, "d2h_bytes_per_step": W * H * 4,
                "ms_per_step": dt / steps * 1e3, "step_ms_min": min(per), "step_ms_median": statistics.median(per),
                "step_ms_max": max(per), "step_ms": [round(x, 2) for x in per]}

    mapped = measure(step_mapped)
    mapped_image = img_host.clone()
    copied = measure(step_copy)
    identical = bool(torch.equal(mapped_image, img_host))
    del host
    return {**mapped, "path": "render kernels read the pinned host buffer over the host link "
                              "(pcr_upload_points_mapped)", "images_identical": identical,
            "copy_path": {**copied, "path": "cudaMemcpyAsync into a device buffer, then render "
                                            "(pcr_upload_points_from_host)"}}


def vertex_order(h, pcr, clouds, dev) -> None:
    """Put every cloud in shuffled-Morton order (Sec. 4), in place: the
    one-time preprocessing the paper prescribes before rendering."""
    import torch
    if not clouds:
        return
    ws = torch.empty(pcr.pcr_reorder_workspace_size(max(c.shape[0] for c in clouds)), dtype=torch.uint8, device=dev)
    for c in clouds:
        pcr.pcr_reorder_morton_shuffle128(h, c, c.shape[0], 0x5EED, pcr.PCR_ORDER_MORTON_SHUFFLE128, ws)
    torch.cuda.synchronize()
    del ws
    torch.cuda.empty_cache()


def run_batched(h, pcr, stream, dev, reps: int) -> dict:
    """8 boxes clouds (1M..200M points) x 8 orbit views (256^2..2048^2), basic
    and HQ frames: every view through the single-view calls (7 launches per
    view) against the batch, tuned (L2 budget and launch configuration) and
    replayed as one CUDA graph; outputs compared bit for bit."""
    import torch
    from paper_2104_07526_gb300 import scenes
    t0 = time.perf_counter()
    clouds = [scenes.boxes(nc, seed=i, device=dev) for i, nc in enumerate(scenes.BATCH_CLOUD_SIZES)]
    vertex_order(h, pcr, clouds, dev)
    views = scenes.batch_views(len(clouds))
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0

    def buffers(W, H):
        npx = W * H
        return {"keys": torch.empty(npx, dtype=torch.int64, device=dev),
                "image": torch.empty(npx, dtype=torch.int32, device=dev),
                "hq_depth": torch.empty(npx, dtype=torch.int32, device=dev),
                "hq_rg": torch.empty(npx, dtype=torch.int64, device=dev),
                "hq_ba": torch.empty(npx, dtype=torch.int64, device=dev),
                "hq_image": torch.empty(npx, dtype=torch.int32, device=dev)}

    per = [buffers(v.width, v.height) for _, v in views]
    bat = [buffers(v.width, v.height) for _, v in views]
    var = pcr.PCR_VARIANT_EARLYZ  # the per-view forms the batch kernels use

    def per_request():
        for (c, v), b in zip(views, per):
            pcr.pcr_upload_points(h, clouds[c], clouds[c].shape[0])
            pcr.pcr_set_matrix(h, v.matrix)
            pcr.pcr_set_viewport(h, v.width, v.height)
            pcr.pcr_set_framebuffer(h, b["keys"], b["hq_depth"], b["hq_rg"], b["hq_ba"])
            pcr.pcr_render_basic(h, var, True)
            pcr.pcr_resolve(h, pcr.PCR_RESOLVE_BASIC, b["image"], 0)
            pcr.pcr_render_hq(h, 1.01, var, True)
            pcr.pcr_resolve(h, pcr.PCR_RESOLVE_HQ, b["hq_image"], 0)

    per_ms = time_loop(per_request, stream, reps=reps, warm=1)
    ws = torch.empty(pcr.pcr_batch_workspace_size(), dtype=torch.uint8, device=dev)
    flags = pcr.PCR_BATCH_BASIC | pcr.PCR_BATCH_HQ
    bclouds = [pcr.batch_cloud(c) for c in clouds]
    bviews = [pcr.batch_view(v.matrix, v.width, v.height, c, flags, **b) for (c, v), b in zip(views, bat)]
    # the tuner's cache: a fresh file, so the first call tunes and the second reads it
    cache = os.path.join(tempfile.gettempdir(), f"pcr_batch_tuning_{os.getpid()}.jsonl")
    if os.path.exists(cache):
        os.remove(cache)
    tuning = pcr.pcr_batch_tune(h, bclouds, bviews, 1.01, 0, ws, cache)
    cached = pcr.pcr_batch_tune(h, bclouds, bviews, 1.01, 0, ws, cache)
    os.remove(cache)
    config = tuning["config"]
    graph = pcr.pcr_batch_capture(h, ws, config)
    try:
        batched_ms = time_loop(lambda: pcr.pcr_graph_launch(h, graph), stream, reps=reps, warm=2)
    finally:
        pcr.pcr_graph_destroy(graph)
    torch.cuda.synchronize()
    identical = all(torch.equal(p_[k], b_[k]) for p_, b_ in zip(per, bat) for k in p_)
    point_views = sum(clouds[c].shape[0] for c, _ in views)
    return {"workload": "8 boxes clouds (1M..200M points, 388M total, shuffled-Morton order) x 8 orbit views "
                        "(256^2..2048^2), basic + HQ",
            "per_request_ms": per_ms, "per_request_launches": 7 * len(views), "batched_graph_ms": batched_ms,
            "batched_launches": pcr.pcr_batch_launch_count(h, ws, config), "speedup": per_ms / batched_ms,
            "identical": identical, "config": config,
            "tuning": {**{k: tuning[k] for k in ("l2_budget_mb", "config", "threads", "unroll1", "unroll2",
                                                 "single_colors", "tried")},
                       "tuned_ms": tuning["best_ms"], "default_ms": tuning["default_ms"],
                       "speedup_over_default": tuning["default_ms"] / tuning["best_ms"],
                       "second_call_from_cache": bool(cached["from_cache"])},
            "point_views_per_s": point_views / (batched_ms * 1e-3), "generate_s": gen_s}


def run_served(h, pcr, stream, dev, seconds: float, max_inflight: int = 3, max_batch_views: int = 64,
               batch_config: int = 0, plain_baseline: bool = True, rates=(2000.0,), streams: int = 3,
               max_batch_clouds: int = 1, policy: int | None = None, max_queue: int = 256,
               deadline_us: int = 0, l2_budget_mb: int = 0) -> list:
    """16 boxes clouds (1M..300M points, shuffled-Morton order) registered
    with the server from host memory, a 150 GB arena, and for each rate a
    Poisson stream of requests (random cloud, resolution 512^2..3840x2160,
    basic or HQ, orbit camera).  The server takes the largest groups of one
    cloud first, 3 batches in flight on 3 streams, and refuses submissions
    beyond 256 queued requests (admission control), so latency stays bounded
    when the offered rate exceeds what the GPU renders.  Latency runs from
    each request's scheduled arrival to its completion.  The same stream is
    then served by plain per-request launches (one request at a time, in
    order, every request).  One result per rate."""
    import torch
    from paper_2104_07526_gb300 import scenes
    sizes = scenes.SERVE_CLOUD_SIZES
    dev_clouds = [scenes.boxes(nc, seed=100 + i, device=dev) for i, nc in enumerate(sizes)]
    vertex_order(h, pcr, dev_clouds, dev)
    host_clouds = [c.cpu().numpy() for c in dev_clouds]
    out = []
    for rate in rates:
        out.append(served_at_rate(h, pcr, dev, dev_clouds, host_clouds, sizes, seconds, rate, max_inflight,
                                  max_batch_views, batch_config, plain_baseline, streams, max_batch_clouds,
                                  pcr.PCR_SERVE_LARGEST_GROUP if policy is None else policy, max_queue,
                                  deadline_us, l2_budget_mb))
    return out


def served_at_rate(h, pcr, dev, dev_clouds, host_clouds, sizes, seconds, rate, max_inflight, max_batch_views,
                   batch_config, plain_baseline, streams, max_batch_clouds, policy=0, max_queue=0,
                   deadline_us=0, l2_budget_mb=0) -> dict:
    import torch
    from paper_2104_07526_gb300 import scenes
    reqs = scenes.serve_requests(int(rate * seconds), rate, seed=7, num_clouds=len(sizes))
    arena = torch.empty(150 << 30, dtype=torch.uint8, device=dev)
    srv = pcr.pcr_server_create(h, arena, 3840, 2160, num_slots=128, max_batch_views=max_batch_views,
                                max_inflight=max_inflight, streams=streams, max_batch_clouds=max_batch_clouds,
                                batch_config=batch_config, depth_factor=1.01, background_rgba=0,
                                max_queue=max_queue, deadline_us=deadline_us, policy=policy,
                                l2_budget_mb=l2_budget_mb)
    try:
        for i, hc in enumerate(host_clouds):
            pcr.pcr_server_add_cloud(srv, i, hc)
        # warm-up: one request per cloud uploads every cloud
        warm = [pcr.pcr_server_submit(srv, i, reqs[0][2], 512, 512, 1) for i in range(len(sizes))]
        left = set(warm)
        while left:
            pcr.pcr_server_step(srv)
            for t in pcr.pcr_server_poll_completed(srv):
                left.discard(t)
                pcr.pcr_server_release(srv, t)
        stats0 = pcr.pcr_server_stats_get(srv)

        def us():
            return time.monotonic_ns() / 1e3  # same clock as the server's steady clock

        t0 = us() + 1000.0
        arrival = [t0 + r[0] * 1e6 for r in reqs]
        lat, pts, last_done, i, done, refused, expired = [], 0, 0.0, 0, 0, 0, 0
        owner = {}
        while done + refused < len(reqs):
            now = us()
            while i < len(reqs) and arrival[i] <= now:
                _, c, m, W, H, flags = reqs[i]
                try:
                    owner[pcr.pcr_server_submit(srv, c, m, W, H, flags)] = i
                except pcr.PcrError as e:  # admission control: the queue is full
                    if e.status != pcr.PCR_ERR_BUSY:
                        raise
                    refused += 1
                i += 1
            pcr.pcr_server_step(srv)
            for t in pcr.pcr_server_poll_completed(srv):
                res = pcr.pcr_server_get_result(srv, t)
                k = owner.pop(t)
                if res.points or res.keys or res.hq_rg:
                    lat.append((res.done_us - arrival[k]) / 1e3)
                    pts += res.points
                    last_done = max(last_done, res.done_us)
                else:  # expired at its deadline, unrendered
                    expired += 1
                pcr.pcr_server_release(srv, t)
                done += 1
        stats = pcr.pcr_server_stats_get(srv)
    finally:
        pcr.pcr_server_destroy(srv)
    span_s = (last_done - arrival[0]) / 1e6
    served = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
              "max_ms": float(np.max(lat)), "completed": len(lat), "refused": refused, "expired": expired,
              "requests_per_s": len(lat) / span_s, "points_per_s": pts / span_s,
              "policy": "largest groups" if policy == pcr.PCR_SERVE_LARGEST_GROUP else "arrival order",
              "max_queue": max_queue, "deadline_ms": deadline_us / 1e3,
              "batches": stats["batches"] - stats0["batches"],
              "mean_batch": (stats["views_launched"] - stats0["views_launched"]) / max(1, stats["batches"] -
                                                                                      stats0["batches"]),
              "uploads": stats["uploads"], "evictions": stats["evictions"], "peak_queue": stats["peak_queue"]}
    del arena
    torch.cuda.empty_cache()
    if not plain_baseline:
        return {"served": served}

    # plain per-request launches on the same arrival schedule
    W0, H0 = 3840, 2160
    fb = pcr.alloc_framebuffer(W0, H0, dev)
    pcr.pcr_set_framebuffer(h, fb["keys"], fb["hq_depth"], fb["hq_rg"], fb["hq_ba"])
    var = pcr.PCR_VARIANT_EARLYZ  # the per-view forms the batch kernels use

    def render(c, m, W, H, flags):
        pcr.pcr_upload_points(h, dev_clouds[c], dev_clouds[c].shape[0])
        pcr.pcr_set_matrix(h, m)
        pcr.pcr_set_viewport(h, W, H)
        if flags & 1:
            pcr.pcr_render_basic(h, var, True)
            pcr.pcr_resolve(h, pcr.PCR_RESOLVE_BASIC, fb["image"], 0)
        else:
            pcr.pcr_render_hq(h, 1.01, var, True)
            pcr.pcr_resolve(h, pcr.PCR_RESOLVE_HQ, fb["image"], 0)

    render(*reqs[0][1:])
    torch.cuda.synchronize()
    t0 = us() + 1000.0
    arrival = [t0 + r[0] * 1e6 for r in reqs]
    lat_p, pts_p = [], 0
    for k, (_, c, m, W, H, flags) in enumerate(reqs):
        while us() < arrival[k]:
            pass
        render(c, m, W, H, flags)
        pcr.pcr_synchronize(h)
        lat_p.append((us() - arrival[k]) / 1e3)
        pts_p += sizes[c]
    span_p = (us() - arrival[0]) / 1e6
    plain = {"p50_ms": float(np.percentile(lat_p, 50)), "p99_ms": float(np.percentile(lat_p, 99)),
             "requests_per_s": len(reqs) / span_p, "points_per_s": pts_p / span_p}
    return {"workload": f"{len(sizes)} boxes clouds ({sizes[0] / 1e6:.0f}M..{sizes[-1] / 1e6:.0f}M points, "
                        "shuffled-Morton order), "
                        f"Poisson {rate:g} requests/s for {seconds:g} s, 512^2..3840x2160, basic/HQ 50/50, "
                        "150 GB arena", "requests": len(reqs), "served": served, "plain": plain,
            "throughput_gain": served["requests_per_s"] / plain["requests_per_s"]}


def run_sweep(h, pcr, orders, views, n, fb, stream) -> dict:
    """Every render variant x vertex order x camera, timed.  Each cell also
    records, compared on the device, whether its exact variants left
    identical buffers: the key buffers of the six exact atomic variants and
    the busy-loop; the colour-payload keys; the HQ buffers of the three HQ
    variants; the HQS1R images against the HQ image; and the depth halves of
    the keys against the original order's for the same camera (any vertex
    order gives the same nearest depths)."""
    import torch
    out = {}
    keys, image = fb["keys"], fb["image"]
    for v in views:
        pcr.pcr_set_matrix(h, v.matrix)
        pcr.pcr_set_viewport(h, v.width, v.height)
        out[v.name] = {}
        depth_ref = None
        for oname, buf in orders.items():
            pcr.pcr_upload_points(h, buf, n)
            row = {}
            same = {"keys": True, "rgb": True, "hq": True, "hq1r_image": True}
            ref = None
            for var in range(7):
                row[pcr.VARIANT_NAMES[var]] = round(time_loop(
                    lambda: pcr.pcr_render_basic(h, var, True), stream, reps=10, warm=2), 4)
                if var == pcr.PCR_VARIANT_ATOMICMIN:
                    ref = keys.clone()
                elif var in pcr.EXACT_VARIANTS:
                    same["keys"] &= bool(torch.equal(keys, ref))
            if depth_ref is None:
                depth_ref = ref >> 32
            else:
                same["depth_vs_first_order"] = bool(torch.equal(ref >> 32, depth_ref))
            rgb_ref = None
            for var in (pcr.PCR_VARIANT_ATOMICMIN, pcr.PCR_VARIANT_EARLYZ, pcr.PCR_VARIANT_DEDUP_EARLYZ):
                row["rgb:" + pcr.VARIANT_NAMES[var]] = round(time_loop(
                    lambda: pcr.pcr_render_rgb(h, var, True), stream, reps=10, warm=2), 4)
                if rgb_ref is None:
                    rgb_ref = keys.clone()
                else:
                    same["rgb"] &= bool(torch.equal(keys, rgb_ref))
            pcr.pcr_last_device_error(h)
            busy = round(time_loop(lambda: pcr.pcr_render_basic(h, pcr.PCR_VARIANT_BUSY_LOOP, True), stream,
                                   reps=5, warm=1), 4)
            # a run whose lock waits ran out dropped points: not a valid time
            if pcr.pcr_last_device_error(h) == 0:
                row["busy-loop"] = busy
                same["busy_loop_keys"] = bool(torch.equal(keys, ref))
            else:
                row["busy-loop"] = "wait limit reached"
            hq_ref = hq_img = None
            for var in (pcr.PCR_VARIANT_ATOMICMIN, pcr.PCR_VARIANT_EARLYZ, pcr.PCR_VARIANT_DEDUP_EARLYZ):
                row["hq:" + pcr.VARIANT_NAMES[var]] = round(time_loop(
                    lambda: pcr.pcr_render_hq(h, 1.01, var, True), stream, reps=5, warm=1), 4)
                got = [fb[k].clone() for k in ("hq_depth", "hq_rg", "hq_ba")]
                if hq_ref is None:
                    hq_ref = got
                    pcr.pcr_resolve(h, pcr.PCR_RESOLVE_HQ, image, 0)
                    hq_img = image.clone()
                else:
                    same["hq"] &= all(bool(torch.equal(a, b)) for a, b in zip(got, hq_ref))
                row["hq1r:" + pcr.VARIANT_NAMES[var]] = round(time_loop(
                    lambda: pcr.pcr_render_hq1r(h, 1.01, var, True), stream, reps=5, warm=1), 4)
                pcr.pcr_resolve(h, pcr.PCR_RESOLVE_HQ1R, image, 0)
                same["hq1r_image"] &= bool(torch.equal(image, hq_img))
            row["identical"] = same
            out[v.name][oname] = row
    return out


ORDER_MODES = {"morton": 0, "morton_shuffle128": 1, "shuffle": 2, "morton63": 3, "morton63_shuffle128": 4}


def run_part(args) -> int:
    """One part alone, through the C ABI, so a profiler sees the library's
    own kernels and little else.  reorder: each order of the scan scene from
    its generation order, run twice (the first warms up), CUDA events.  batch:
    the 8 boxes clouds x 8 orbit views (shuffled-Morton order, basic + HQ),
    prepared once and launched four times with configuration 0.  served: the
    served workload's Poisson stream at 8000 requests/s for --served-seconds
    through the server, without the plain-launch arm."""
    import torch
    from paper_2104_07526_gb300 import build as lib_build
    from paper_2104_07526_gb300 import pcr, scenes
    lib_build.build()
    stream = torch.cuda.current_stream()
    ctx = pcr.Context(0, stream=stream)
    h = ctx.handle
    out = {}
    if args.part == "reorder":
        n = args.points
        cloud = scenes.scan(n, seed=0, device="cuda")
        ws = torch.empty(pcr.pcr_reorder_workspace_size(n), dtype=torch.uint8, device="cuda")
        for name in args.orders.split(","):
            best = None
            for _ in range(2):
                buf = cloud.clone()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record(stream)
                pcr.pcr_reorder_morton_shuffle128(h, buf, n, 0x5EED, ORDER_MODES[name], ws)
                b.record(stream)
                torch.cuda.synchronize()
                best = a.elapsed_time(b) if best is None else min(best, a.elapsed_time(b))
                del buf
            out[name] = round(best, 3)
    elif args.part == "served":
        out["served"] = run_served(h, pcr, stream, "cuda", args.served_seconds, plain_baseline=False,
                                   rates=(8000.0,))[0]["served"]
    else:
        clouds = [scenes.boxes(nc, seed=i, device="cuda") for i, nc in enumerate(scenes.BATCH_CLOUD_SIZES)]
        vertex_order(h, pcr, clouds, "cuda")
        views = scenes.batch_views(len(clouds))
        bufs = [{k: torch.empty(v.width * v.height, dtype=t, device="cuda") for k, t in
                 (("keys", torch.int64), ("image", torch.int32), ("hq_depth", torch.int32), ("hq_rg", torch.int64),
                  ("hq_ba", torch.int64), ("hq_image", torch.int32))} for _, v in views]
        flags = pcr.PCR_BATCH_BASIC | pcr.PCR_BATCH_HQ
        ws = torch.empty(pcr.pcr_batch_workspace_size(), dtype=torch.uint8, device="cuda")
        pcr.pcr_batch_prepare(h, [pcr.batch_cloud(c) for c in clouds],
                              [pcr.batch_view(v.matrix, v.width, v.height, c, flags, **b) for (c, v), b in
                               zip(views, bufs)], 1.01, 0, ws)
        times = []
        for _ in range(4):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pcr.pcr_batch_launch(h, ws, 0)
            b.record(stream)
            torch.cuda.synchronize()
            times.append(round(a.elapsed_time(b), 3))
        out["batch_ms"] = times
    ctx.close()
    print(json.dumps({"part": args.part, **out}), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    cfg = CONFIGS[args.config]
    if args.part:
        return run_part(args)
    if args.impl == "reference":
        return run_reference(args, cfg)
    return run_ours(args, cfg)


if __name__ == "__main__":
    sys.exit(main())
