"""The benchmark's roofline arithmetic on CPU: the algorithmic bytes of the dominant stages follow the
per-unit figures of the design notes, the DRAM traffic is reported only while the kernel sources match the
ncu capture it came from, and the summary carries the figures it names."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

COUNTS = dict(V=50010, F=100016, npx=640 * 480, NP=56, nvis=15114, nassoc_px=17000, nA=9000, n_valid_px=17000,
              nblk=150)


def test_association_bytes_are_the_scope_figure():
    # 4 B depth + 4 B correspondence per pixel, 28 B per associated vertex (its sums)
    kind, b = bench.algorithmic("associate", **COUNTS)
    assert kind == "hbm" and b == 640 * 480 * 8 + 9000 * 28


def test_streaming_stage_bytes_per_unit():
    c = dict(COUNTS)
    kind, skin = bench.algorithmic("skin", **c)
    assert kind == "hbm" and skin == c["V"] * 100 + c["npx"] * 16
    kind, red = bench.algorithmic("reduce", **c)
    assert red == c["nblk"] * 56 * 56 * 4 + 56 * 56 * 8
    kind, ev = bench.algorithmic("lm_eval", **c)
    assert ev == c["nA"] * 64 + c["nblk"] * 4
    # each stage grows with its own units only
    c2 = dict(c, V=2 * c["V"])
    assert bench.algorithmic("skin", **c2)[1] - skin == c["V"] * 100
    assert bench.algorithmic("associate", **c2)[1] == bench.algorithmic("associate", **c)[1]
    kind, fl = bench.algorithmic("lm_solve", **c)
    assert kind == "fp64" and fl == 6 * (55 ** 3 / 3.0 + 2 * 55 * 55)
    assert bench.algorithmic("no such stage", **c) == (None, 0)


def test_traffic_only_from_a_capture_of_the_current_kernels():
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        t = json.load(f)
    cur = bench.kernel_source_hash()
    for name, e in t["kernels"].items():
        got = bench.ncu_traffic(name)
        if e.get("kernel_source_hash", t.get("kernel_source_hash")) == cur:
            assert got == e.get("dram_bytes_per_launch_full_size")
        else:
            assert got is None
    assert bench.ncu_traffic("no such kernel") is None


def test_summary_names_its_figures():
    line = {"value": 5000.0, "plain": {"value": 700.0}, "e2e": {"value": 4000.0}, "latency_ms": {"p99": 12.0},
            "roofline": {"frac": 0.1, "kernel": "associate"},
            "precision": {"fp32": {"serving_fps": 4900.0, "latency_ms": {"p99": 26.0},
                                   "lockstep_vs_oracle": {"theta_rad_max": 1e-6, "offsets_mm_max": 1e-3,
                                                          "energy_rel_max_matched": 1e-6, "nontie_mismatches": 0,
                                                          "lm_decisions_equal": True, "frames": 2}}},
            "admission_serving": {"budget_bytes": 1, "peak_device_bytes_in_use": 1, "achieved_fps": 2.0, "x": 3}}
    s = bench.summary_of(line)
    assert s["plain_fps"] == 700.0 and s["batched_fps"] == 5000.0 and s["e2e_fps"] == 4000.0
    assert s["latency_p99_ms"] == 12.0 and s["roofline_frac"] == 0.1 and s["roofline_kernel"] == "associate"
    assert s["serving_fps"] == {"fp32": 4900.0} and s["serving_p99_ms"] == {"fp32": 26.0}
    assert s["lockstep_vs_oracle"]["fp32"]["nontie_mismatches"] == 0
    assert "frames" not in s["lockstep_vs_oracle"]["fp32"]
    assert s["admission"] == {"budget_bytes": 1, "peak_device_bytes_in_use": 1, "achieved_fps": 2.0}
    # a line without the optional parts still summarises
    assert bench.summary_of({"value": 1.0})["batched_fps"] == 1.0
