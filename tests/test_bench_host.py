"""Host-side parts of bench.py's CPU baseline: the oracle timed on all host
cores and on one (the thread count is restored afterwards), and the host's
CPU description."""
import os
import sys

import oracle as O
from paper_0802_2488_gb300 import inputs

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_cpu_baseline_reports_all_cores_and_one():
    before = O.threads()
    r = bench.cpu_baseline([inputs.config1()], budget_s=0.2, single_s=0.1)
    assert O.threads() == before
    assert r["kind"] == "oracle" and r["cores"] == before and r["value"] > 0
    assert r["single_thread"]["cores"] == 1 and r["single_thread"]["value"] > 0
    assert r["host"]["nproc"] == os.cpu_count() and r["host"]["cpu"]


def test_oracle_thread_control():
    n = O.threads()
    try:
        O.set_threads(1)
        assert O.threads() == 1
    finally:
        O.set_threads(n)
    assert O.threads() == n


def test_clock_summary_parses_nvidia_smi_rows():
    """Median SM clock under load, the maximum, and the throttle reasons seen
    active in any sample (the bench line's `clocks`)."""
    s = bench.ClockSampler(0)
    rows = [
        "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1965, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    s.f.write("\n".join(rows) + "\n")
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 4
    assert not os.path.exists(s.f.name)


def test_clock_summary_without_samples():
    s = bench.ClockSampler(0)
    out = s.summary()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_workload_configs():
    """The bench's workloads are the stated configurations, named by what
    they are, with the iteration cap in the config block."""
    for name, L, n, n_inc in (("c1", 64, 1, 20), ("c2", 256, 1, 40), ("c3", 512, 64, 30), ("c4", 4096, 1, 50)):
        probs, cfg = bench.workload(name, 77)
        assert len(probs) == n and cfg["L"] == L and cfg["n_solves"] == n and cfg["n_inc"] == n_inc
        assert cfg["max_iter_per_increment"] == 77 and cfg["tol"] == 1e-8
        assert "at most 77 iterations" in cfg["workload"] and f"L={L}" in cfg["workload"]
