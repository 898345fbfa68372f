"""Host logic of bench.py that needs no GPU: the clock record of the timed
region, the rule that ncu traffic counters are reported only while the
profiled sources are unchanged, and the lambda thresholds of the workload."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler(rows):
    c = bench.ClockSampler(0)
    c.samples = [[x.strip() for x in r.split(",")] for r in rows]
    return c


def test_clock_summary_median_max_and_reasons():
    rows = ["2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "2055, 2070, 1200.0, 0x4, Not Active, Not Active, Not Active, Active",
            "2070, 2070, 1250.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "1500, 2070, 1300.0, 0x8, Active, Not Active, Not Active, Not Active"]
    c = _sampler(rows)
    s = c.summary(0, 2)  # the timed region: samples 0..2
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    s = c.summary(1, 3)
    assert s["sm_mhz"] == 2055  # median of 2055, 2070, 1500
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_summary_without_samples_or_values():
    assert _sampler([]).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
    s = _sampler(["[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]"]).summary()
    assert s["sm_mhz"] is None and s["sm_max_mhz"] is None and s["reasons"] == []
    # an empty window falls back to the last sample
    s = _sampler(["1980, 2070, 1.0, 0x0, Not Active, Not Active, Active, Not Active"]).summary(5, 9)
    assert s["sm_mhz"] == 1980 and s["reasons"] == ["sw_thermal_slowdown"]


def test_profiled_counters_follow_the_sources(tmp_path, monkeypatch):
    import hashlib

    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    sha = hashlib.sha1(src.read_bytes()).hexdigest()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "PROFILED", {"x": {"src": {"k.cu": sha}, "dram_bytes": 123}})
    assert bench.profiled("x")["dram_bytes"] == 123
    src.write_text("__global__ void k() { }\n")  # any change of the source drops the counters
    assert bench.profiled("x") is None
    monkeypatch.setattr(bench, "PROFILED", {"x": {"src": {"missing.cu": sha}, "dram_bytes": 1}})
    assert bench.profiled("x") is None


def test_lambda_thresholds_match_the_oracle_convention(orc):
    rng = np.random.default_rng(4)
    A = [rng.standard_normal((s, 6)) for s in (9, 8, 7)]
    hi, lo = bench.lam_thresholds(A)
    ohi, olo = orc.default_lambda(A)
    assert abs(hi - ohi) <= 1e-12 * ohi and abs(lo - olo) <= 1e-12 * olo
    assert abs(hi / lo - 1e6) <= 1e-6
