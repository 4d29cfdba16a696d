"""Host helpers of bench.py that shape the reported numbers, on CPU: the DRAM
traffic record (profiles/ncu_traffic.json) is scaled to a launch's frames
and dropped once a source it was taken from changes; the clock record is
summarised from nvidia-smi's CSV lines (median SM clock, the throttle
reasons seen, unsampled when nothing came back)."""

import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _record():
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        return json.load(f)


def test_traffic_record_scales_to_the_launch_frames():
    rec = _record()
    for stage, k in rec["kernels"].items():
        per_frame = (k["dram_read_bytes"] + k["dram_write_bytes"]) / k["frames"]
        got = bench.ncu_traffic(stage, 64)
        if got is None:  # a source changed since the capture: nothing to scale
            continue
        assert got == pytest.approx(per_frame * 64)
    assert bench.ncu_traffic("no_such_stage", 64) is None


def test_traffic_record_dropped_when_a_source_changes(tmp_path, monkeypatch):
    rec = _record()
    srcs = sorted({s for k in rec["kernels"].values() for s in k["sources"]})
    for s in srcs + ["profiles/ncu_traffic.json"]:
        dst = tmp_path / s
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copyfile(os.path.join(ROOT, s), dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    before = {st: bench.ncu_traffic(st, 8) for st in rec["kernels"]}
    # one byte more in the texture kernel's own source
    tex = rec["kernels"]["texture"]["sources"][0]
    with open(tmp_path / tex, "a") as f:
        f.write("\n")
    after = {st: bench.ncu_traffic(st, 8) for st in rec["kernels"]}
    assert after["texture"] is None
    for st, k in rec["kernels"].items():
        if tex not in k["sources"]:
            assert after[st] == before[st]


def test_clock_summary():
    cs = bench.ClockSampler(0)
    cs.out = "\n".join([
        "2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 950.0, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1000.5, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ])
    s = cs.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    cs.out = ""
    assert cs.summary()["reasons"] == ["unsampled"]


def test_throughput_counts_every_rank():
    assert bench.job_throughput(64 * 10, 1, 0.5) == pytest.approx(1280.0)
    assert bench.job_throughput(64 * 10, 4, 0.5) == pytest.approx(4 * 1280.0)
