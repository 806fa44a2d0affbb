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


def test_convergence_summary_counts_what_increments_reached():
    """The bench reports how many increments met the tolerances before the
    cap and the indicators they stopped at; solves/s "at tol" needs all."""
    import numpy as np
    from paper_0802_2488_gb300 import binding as B
    a = np.zeros(3, dtype=B.RECORD_DTYPE)
    a["status"] = [0, 1, 1]
    a["eta1"] = [5e-9, 2e-5, 1e-4]
    a["eta2"] = [1e-9, 1e-9, 3e-9]
    a["iterations"] = [40, 100, 100]
    b = np.zeros(2, dtype=B.RECORD_DTYPE)
    b["status"] = [0, 2]
    b["eta1"] = [1e-9, 1e-9]
    b["iterations"] = [10, 50]
    c = bench.convergence([a, b])
    assert c["increments"] == 5 and c["converged"] == 2 and c["capped"] == 2 and c["numeric_failures"] == 1
    assert c["eta1_max"] == 1e-4 and c["eta1_median"] == 5e-9 and c["eta2_max"] == 3e-9
    assert c["iterations_per_increment_mean"] == 60.0


def test_roofline_uses_the_algorithmic_work_of_each_pass():
    """FP32: 73 B per pixel in the row pass and 24 B in the column pass over
    the mean launch time, against the HBM peak; FP64: 15 log2 L + 60 and
    15 log2 L + 25 flops per pixel against the FP64 peak; the dominant pass
    is the longer one."""
    r = bench.roofline("fp32", 512, 64, 0.184, 0.337, 6770.0, "measured", 0)
    n = 512 * 512 * 64
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["kernel"] == "row_pass<float,512,0>"
    assert r["passes"]["col"]["kernel"] == "col_pass_rs<512>"
    assert abs(r["achieved"] - 73 * n / 0.337e-3 / 1e9) < 1e-6
    assert abs(r["passes"]["col"]["achieved"] - 24 * n / 0.184e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6770.0) < 1e-12
    # traffic only where an ncu capture of that kernel at that launch shape
    # exists, and only while the kernel sources are those it ran
    e = bench.TRAFFIC[("fp32", 512, 64, 0, "row")]
    if bench.kernel_source_digest(bench.PASS_HEADERS) == e[2]:
        assert r["traffic"] == e[0]
    else:
        assert r["traffic"] is None
    assert bench.roofline("fp32", 512, 64, 0.184, 0.337, 6770.0, "measured", 1)["traffic"] is None
    assert bench.roofline("fp32", 512, 16, 0.184, 0.337, 6770.0, "measured", 0)["traffic"] is None
    r4 = bench.roofline("fp32", 4096, 1, 0.15, 0.47, 6770.0, "measured", 2)
    assert r4["kernel"] == "row_pass_rs<4096>"
    rd = bench.roofline("fp32_defect", 512, 64, 0.12, 0.58, 6770.0, "measured", 0)
    assert rd["bound"] == "hbm" and rd["kernel"] == "row_pass_dc<512,0>"
    assert abs(rd["achieved"] - 113 * n / 0.58e-3 / 1e9) < 1e-6
    ed = bench.TRAFFIC[("fp32_defect", 512, 64, 0, "row")]
    assert rd["traffic"] == (ed[0] if bench.kernel_source_digest(bench.DEFECT_HEADERS) == ed[2] else None)
    r = bench.roofline("fp64", 256, 1, 0.040, 0.030, 1.25, "measured", 1)
    assert r["bound"] == "alu" and r["kernel"] == "col_pass<double,256,1>" and r["traffic"] is None
    assert abs(r["achieved"] - (15 * 8 + 25) * 65536 / 0.040e-3 / 1e12) < 1e-12
    assert abs(r["passes"]["row"]["achieved"] - (15 * 8 + 60) * 65536 / 0.030e-3 / 1e12) < 1e-12


def test_traffic_reads_null_once_the_kernel_sources_change(monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC", {k: (v[0], v[1], "0" * 16) for k, v in bench.TRAFFIC.items()})
    r = bench.roofline("fp32", 512, 64, 0.184, 0.337, 6770.0, "measured", 0)
    assert r["traffic"] is None and "changed" in r["traffic_note"]
    assert all(p["traffic"] is None for p in r["passes"].values())


def test_traffic_entries_match_their_profile_summaries():
    """Every traffic figure the benchmark can report names a committed ncu
    summary under profiles/ that states the same kernel-header digest and the
    same DRAM bytes per launch (in MB, as the launch list prints them)."""
    import os
    for key, (nbytes, path, digest) in bench.TRAFFIC.items():
        full = os.path.join(bench.ROOT, path)
        assert path.startswith("profiles/") and os.path.isfile(full), key
        text = open(full).read()
        assert digest in text, (key, digest)
        assert f"{nbytes / 1e6:.1f} MB" in text, (key, nbytes)
