"""Host logic of bench.py (no GPU): the workload defaults of the bench line,
the roofline entry built from the engine's counters, and the committed ncu
traffic records it scales."""

import json
import os
import types

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _args(**kw):
    base = dict(requests=None, work_budget=None, frontier_cap_gib=None)
    base.update(kw)
    return types.SimpleNamespace(**base)


def test_workload_defaults():
    big = bench.workload_settings("boards256", _args())
    assert big["requests"] == 3000 and big["work_budget"] == 1 << 16
    assert big["flags"] & 2 and big["mode"] == 0 and big["frontier_cap"] == 16 << 30
    small = bench.workload_settings("regular32", _args())
    assert small["work_budget"] == 0 and small["flags"] == 0 and small["requests"] is None
    assert bench.workload_settings("boards256", _args(work_budget=7))["work_budget"] == 7
    assert bench.line_unit("boards256") == "decisions/s" and bench.line_unit("regular32") == "embeddings/s"


def _run(name, tail_ms, expand_ms, roof_ms=2.0, steps=2):
    stats = {"tail_ms": tail_ms * steps, "expand_ms": expand_ms * steps, "expand_launches": 10 * steps,
             "expand_bytes": 4.0e8 * steps, "tail_launches": 3 * steps, "tail_int_ops": 3.0e9 * steps,
             "tail_parents": 6.0e6 * steps}
    return {"stats_roof": stats, "roof_steps": steps, "roof_ms": [roof_ms] * steps,
            "wl": types.SimpleNamespace(name=name), "nreq": 10000}


def test_roofline_takes_the_larger_share():
    peaks = {"hbm_gbs": 6000.0}
    int_peak = {"mix_gops": 15000.0, "source": "test"}
    r = bench.roofline(_run("boards256", tail_ms=0.1, expand_ms=1.5), peaks, "measured", int_peak)
    assert r["bound"] == "hbm"
    # 10 launches per step of 4e7 algorithmic bytes each in 0.15 ms
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(4.0e7)
    assert r["achieved"] == pytest.approx(4.0e7 / 0.15e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0)
    assert r["share_of_step"] == pytest.approx(0.75)
    t = bench.roofline(_run("regular32", tail_ms=1.2, expand_ms=0.4), peaks, "measured", int_peak)
    assert t["bound"] == "alu" and t["peak"] == 15000.0
    # 3 launches per step of 1e9 operations each in 0.4 ms
    assert t["achieved"] == pytest.approx(1.0e9 / 0.4e-3 / 1e9)


def test_traffic_records_scale_and_check_their_sources():
    for name, field in (("k_expand_traffic.json", "dram_bytes_per_algorithmic_byte"),
                        ("k_last_traffic.json", "dram_bytes_per_parent")):
        with open(os.path.join(ROOT, "profiles", name)) as f:
            rec = json.load(f)
        assert rec[field] > 0 and rec["command"].startswith("ncu ") and "bench.py" in rec["command"]
        assert len(rec["source_sha256_16"]) == 16 and rec["workload"]
    with open(os.path.join(ROOT, "profiles", "k_expand_traffic.json")) as f:
        rec = json.load(f)
    if rec["source_sha256_16"] == bench._kernel_source_hash():
        got = bench._expand_traffic_per_launch("boards256", 1.0e8)
        assert got == pytest.approx(rec["dram_bytes_per_algorithmic_byte"] * 1.0e8)
    assert bench._expand_traffic_per_launch("regular32", 1.0e8) is None  # another workload's record
