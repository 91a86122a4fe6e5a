"""Host helpers of the benchmark (no GPU): the clock record that decides
whether a run is kept, the DRAM-traffic lookup tied to the kernel source, and
the byte model's inputs."""
import json
import os

import numpy as np
import pytest

import bench
from paper_2603_25068_b300 import scenario as S


def _sampler(lines):
    c = bench.ClockSampler(0)
    c.lines = lines
    return c.summary()


def test_clock_summary_reports_median_max_and_reasons():
    ok = "0, 2032, 2032, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1900, 2032, 1100.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2032, 1100.0, 0x0000000000000020, Not Active, Active, Not Active, Not Active"
    s = _sampler([ok, ok, capped])
    assert s["sm_mhz"] == 2032.0 and s["sm_max_mhz"] == 2032.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]                   # kept and noted
    s = _sampler([ok, hot, "garbage", ""])
    assert s["samples"] == 2 and s["reasons"] == ["hw_thermal_slowdown"]   # a rejected run
    assert _sampler([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_traffic_record_is_tied_to_the_kernel_source(monkeypatch):
    p = os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")
    e = json.load(open(p))["k_persist"]["city_1M"]
    units = e["units_per_launch"]
    if e["source_hash"] == bench.source_hash():
        assert bench.ncu_traffic("k_persist", "city_1M", units) == pytest.approx(e["dram_bytes_per_launch"])
        # a smaller launch scales by the units it processes
        assert bench.ncu_traffic("k_persist", "city_1M", units / 4) == pytest.approx(e["dram_bytes_per_launch"] / 4)
    monkeypatch.setattr(bench, "source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic("k_persist", "city_1M", units) is None      # stale counters are not reported
    assert bench.ncu_traffic("k_nothing", "city_1M", units) is None


def test_choice_degree_excludes_the_u_turn():
    # a chain 0 -> 1 -> 2 -> 3 with return links: after a link the only choices
    # are onward (or back, at the chain's end, where it is the only one)
    sc = S.line_network(n_links=3)
    d = bench.avg_choice_degree(sc)
    # heads of the 6 links: 1, 2, 3 (forward) and 0, 1, 2 (backward); out-degrees
    # 2, 2, 1, 1, 2, 2; minus the U-turn where another choice remains
    assert d == pytest.approx(np.mean([1, 1, 1, 1, 1, 1]))


def test_byte_model_terms():
    sc = S.tiny_grid()
    assert bench.kernel_a_bytes(sc, 0, 0, 3.0) == 32.0 * sc.L + 8.0 * sc.V
    assert bench.kernel_a_bytes(sc, 10, 2, 3.0) - bench.kernel_a_bytes(sc, 0, 0, 3.0) == 8.0 * 10 + (60 + 72) * 2
