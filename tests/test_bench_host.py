"""Host-side logic of bench.py that shapes its JSON line: the traffic record
that is reported only while it matches the kernel sources, the reorder
roofline arithmetic, the CPU sample, the workload description and the
command-line defaults the timing rules require."""
import hashlib
import os
import sys

import pytest

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _write_record(root, sources, variant="early-z", points=100_000_000, bytes_per_launch=1600300000):
    h = hashlib.sha256()
    for p in sources:
        with open(p, "rb") as f:
            h.update(f.read())
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    with open(os.path.join(root, "profiles", bench.TRAFFIC_RECORD), "w") as f:
        f.write("# a comment line = with an equals sign\n")
        f.write(f"sources_sha256={h.hexdigest()}\nvariant={variant}\npoints={points}\n"
                f"bytes_per_launch={bytes_per_launch}\nnote=test record\n")


def test_traffic_record_follows_sources_and_scales(tmp_path, monkeypatch):
    srcs = []
    for name, text in (("a.cu", "kernel a\n"), ("b.cuh", "helper b\n")):
        p = tmp_path / name
        p.write_text(text)
        srcs.append(str(p))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic(srcs, "early-z", 800_000_000) is None  # no record yet
    _write_record(str(tmp_path), srcs)
    rec = bench.recorded_traffic(srcs, "early-z", 800_000_000)
    assert rec["bytes_per_launch"] == pytest.approx(8 * 1600300000.0)  # scaled by the points
    assert rec["captured_points"] == 100_000_000 and rec["note"] == "test record"
    assert bench.recorded_traffic(srcs, "early-z", 100_000_000)["bytes_per_launch"] == pytest.approx(1600300000.0)
    assert bench.recorded_traffic(srcs, "dedup+early-z", 800_000_000) is None  # another variant was timed
    (tmp_path / "b.cuh").write_text("helper b changed\n")
    assert bench.recorded_traffic(srcs, "early-z", 800_000_000) is None  # the kernel changed since the capture


def test_committed_traffic_record_is_for_the_timed_variant():
    path = os.path.join(ROOT, "profiles", bench.TRAFFIC_RECORD)
    if not os.path.exists(path):
        pytest.skip("no traffic record for the current kernels")
    with open(path) as f:
        kv = dict(line.split("=", 1) for line in f.read().splitlines() if "=" in line and not line.startswith("#"))
    assert kv["variant"].strip() == bench.HEADLINE_VARIANT
    per_point = float(kv["bytes_per_launch"]) / int(kv["points"])
    assert 16.0 <= per_point < 16.2  # 16 B per point, plus little


def test_reorder_roofline_arithmetic():
    alg = bench.REORDER_ALGORITHMIC_BYTES_PER_POINT
    assert alg["morton"] == alg["morton_shuffle128"] == 128 and alg["shuffle"] == 104
    assert alg["morton63"] == alg["morton63_shuffle128"] == 192
    table = bench.REORDER_BYTES_PER_POINT
    assert table["morton"] == 148 and table["morton_shuffle128"] == 149 and table["shuffle"] == 172
    assert table["morton63"] == 276 and table["morton63_shuffle128"] == 277
    n, peak = 800_000_000, 6760.9
    out = bench.reorder_roofline({"morton": 27.5, "shuffle": 48.0}, n, peak)
    assert out["morton"]["algorithmic_gb"] == pytest.approx(102.4)
    assert out["morton"]["achieved_gbs"] == pytest.approx(102.4 / 27.5e-3)
    assert out["morton"]["design_over_algorithmic"] == pytest.approx(148 / 128)
    assert out["shuffle"]["frac"] == pytest.approx(83.2 / 48.0e-3 / peak)


def test_cpu_sample_and_its_description():
    assert bench.cpu_sample_indices(10, 3).tolist() == [0, 3, 6]
    assert bench.cpu_sample_indices(5, 10).tolist() == [0, 1, 2, 3, 4]
    assert bench.describe_sample(5, 5) == "the first 5 of the 5 points"
    assert bench.describe_sample(800, 100) == "every 8th point of the 800-point cloud (100 points)"


class _View:
    def __init__(self, name, w, h):
        self.name, self.width, self.height = name, w, h


def test_workload_config_names_the_timed_variant_and_cache_case():
    big = bench.workload_config(bench.CONFIGS["scan800M"], _View("overview", 1920, 1080), "dedup+early-z")
    assert big["variant"] == "dedup+early-z" and "basic frame with dedup+early-z" in big["workload"]
    assert big["points"] == 800_000_000 and big["l2"].startswith("inputs larger than L2")
    small = bench.workload_config(bench.CONFIGS["sphere1M"], _View("front", 640, 480), bench.HEADLINE_VARIANT)
    assert small["l2"].startswith("inputs fit in L2")


def test_default_arguments_meet_the_timing_rules():
    args = bench.parse_args([])
    assert args.gpus == 1 and args.impl == "ours" and args.config == "scan800M"
    assert args.warmup >= 3 and args.steps >= 50
    assert bench.HQ_VARIANT in ("early-z", "dedup+early-z")


def test_sections_at_one_and_several_gpus():
    args = bench.parse_args([])
    one = bench.sections(args, 1)
    assert all(one.values())
    many = bench.sections(args, 4)
    assert many["hq"] and many["e2e"]
    assert not any(many[k] for k in ("sweep", "batched", "small", "served", "cpu"))
    quiet = bench.sections(bench.parse_args(["--no-hq", "--no-e2e", "--no-served", "--no-cpu"]), 1)
    assert not quiet["hq"] and not quiet["e2e"] and not quiet["served"] and not quiet["cpu"]
    assert quiet["sweep"] and quiet["batched"] and quiet["small"]
