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
