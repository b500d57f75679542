"""Host logic of the benchmark (no GPU): the clock record taken during the timed
region, and the whole-job rate of independent replicas."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _row(sm, mx, hw="Not Active", hw_th="Not Active", sw_th="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, 812.35, 0x0000000000000000, {hw}, {hw_th}, {sw_th}, {cap}\n"


def test_clock_summary_median_max_and_reasons():
    lines = [_row(2070, 2070), _row(1995, 2070, cap="Active"), _row(2040, 2070), "garbage\n",
             _row("[N/A]", 2070)]
    c = bench.summarize_clocks(lines)
    assert c["samples"] == 4
    assert c["sm_mhz"] == pytest.approx(2040.0)     # median of 2070, 1995, 2040
    assert c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_every_throttle_kind():
    lines = [_row(1400, 2070, hw="Active"), _row(1400, 2070, hw_th="Active"), _row(1400, 2070, sw_th="Active")]
    assert bench.summarize_clocks(lines)["reasons"] == ["hw_slowdown", "hw_thermal_slowdown",
                                                        "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    c = bench.summarize_clocks([])
    assert c == {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}


def test_job_rate_counts_every_rank():
    # 4 replicas, 1,432 buses x 20,000 steps each, slowest rank 100 ms
    assert bench.job_rate(1432 * 20000, 4, 100.0) == pytest.approx(4 * 1432 * 20000 / 0.1)
