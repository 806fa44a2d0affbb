#!/usr/bin/env python3
"""Throughput of the augmented-Lagrangian FFT solve (Willot & Pellegrini,
arXiv:0802.2488) on one GB300, printed as one JSON line.

Headline (the default workload): the batched FP32 form.  A step is one
batched solve of 64 realizations of an L = 512 lattice (i.i.d. Bernoulli
voids f in {0.05, 0.10, 0.20, 0.30} x seeds 0-15; seeds 0-7 equibiaxial to
2x the void-free yield strain, 8-15 shear to 3x), 30 increments each, all
advanced together in one device-driven loop, equilibrium and macro
tolerances 1e-8, each increment capped at --cap iterations; the masks are
generated and the plastic clusters of every increment labelled.  `value`
counts the pixel-iterations the method ran (sum over solves and increments
of L^2 x iterations) per second of device time with the inputs in HBM;
`e2e` is the same through the C ABI with host buffers (pinned masks in;
records, final strain, plastic flags and cluster labels out) and the copies
inside the timed region.  `convergence` gives what each increment reached
(eta1, eta2 and how many increments met the tolerances before the cap);
solves/s "at tol" is reported only when every increment converged.

A single-GPU default run adds sub-objects measured in the same process:
  c4   the L = 4096, f = 0.35 lattice (FP32), with both passes' HBM roofline;
  c5   the serving stream (Poisson arrivals, L in {128..1024}): p50/p99
       latency and solves/s through submit / serve_step / poll;
  c2   the L = 256 shear lattice in plain FP64 (FP64-ALU roofline against the
       measured FP64 peak), its FP32 form with the field and curve errors
       against FP64, and plain FP64 against the mixed-precision solve and
       the defect-correction form at a tolerance all reach;
  batched_at_tol  8 lattices of the batched recipe at tol 1e-8 in one call:
       plain FP64 against the defect-correction form.

--impl reference times the oracle (the plain FP64 CPU implementation) on
this machine's host cores on a bounded sample of the same workload.

Multi-GPU (torchrun): every rank solves its own copy (replicas, no
collective); value = all ranks' pixel-iterations / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("pixel-iterations/s and solves/s at equilibrium tol 1e-8 (FP32 batched vs FP64 plain); p50/p99")
UNIT = "pixel-iterations/s"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="epfft", choices=["epfft", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3", "c4", "c5"])
    ap.add_argument("--requests", type=int, default=150, help="c5: requests in the stream")
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32", "fp32_defect"],
                    help="default: fp64 for c1/c2, fp32 for c3/c4/c5")
    ap.add_argument("--cap", type=int, default=None, help="max iterations per increment")
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the c4 / c5 / c2 sub-objects of a single-GPU default run")
    a = ap.parse_args()
    if a.precision is None:
        a.precision = "fp64" if a.workload in ("c1", "c2") else "fp32"
    if a.cap is None:
        a.cap = CAPS[a.workload]
    return a


# iterations per increment at most, per workload (the AL needs O(10^3) and
# more per increment on these lattices, see the convergence objects)
CAPS = {"c1": 2000, "c2": 300, "c3": 100, "c4": 60, "c5": 20}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(vals, device=None):
    """Elementwise maximum of the floats `vals` over the ranks of the default
    process group (the slowest replica's times); the values themselves when
    there is one rank or no group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in vals]
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_value(ws: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput of ws replicas of the same workload: the units
    all ranks processed over the slowest rank's time."""
    return ws * units_per_rank / seconds


def workload(name: str, cap: int):
    """The problems of one step and the config block of the JSON line."""
    from paper_0802_2488_gb300 import inputs
    if name == "c3":
        probs = inputs.config3()
        desc = ("64 realizations of L=512 (f in {0.05,0.10,0.20,0.30} x seeds 0-15; seeds 0-7 equibiaxial to "
                "2x yield, 8-15 shear to 3x yield), 30 increments each, advanced together in one device loop")
    else:
        P = {"c1": inputs.config1, "c2": inputs.config2, "c4": inputs.config4}[name]()
        probs = [P]
        desc = (f"{P.name}: L={P.L}, f={P.f:.2f} Bernoulli voids (seed {P.seed}), {P.mode} to "
                f"{P.multiple:g}x yield in {P.n_inc} increments")
    cfg = dict(workload=f"{desc}; mu=1 lambda=1.5 Y=1, C0=matrix, tol 1e-8 (eta1, eta2), at most {cap} "
                        f"iterations per increment, plastic clusters labelled per increment",
               L=probs[0].L, n_solves=len(probs), n_inc=[p.n_inc for p in probs][0] if len(probs) == 1 else 30,
               max_iter_per_increment=cap, tol=1e-8)
    return probs, cfg


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def host_cpu() -> str:
    """CPU model of this host (first 'model name' of /proc/cpuinfo, else the
    platform's processor string)."""
    import platform
    arm = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":", 1)[0].strip().lower()
                if key in ("model name", "cpu model"):
                    return line.split(":", 1)[1].strip()
                if key in ("cpu implementer", "cpu part") and key not in arm:
                    arm[key] = line.split(":", 1)[1].strip()
    except OSError:
        pass
    if arm:  # Arm hosts name the core by implementer and part number
        return f"{platform.machine()} (implementer {arm.get('cpu implementer')}, part {arm.get('cpu part')})"
    return platform.processor() or platform.machine()


def cpu_baseline(probs, budget_s: float = 15.0, single_s: float = 3.0):
    """The oracle as it stands, on this machine's host cores (OpenMP over all
    of them, and on one), on a bounded sample of the workload: the first
    increment of the first problem of the workload, with as many iterations
    as fit in ~budget_s (~single_s on one core)."""
    import oracle as O
    P = probs[0]
    mask = O.mask(P.L, P.f, P.seed)
    mat = O.material()
    O.build()

    def timed(seconds):
        t = time.perf_counter()
        O.solve(mask, mat, P.path[:1], max_iter=2)
        per_it = (time.perf_counter() - t) / 2
        n_it = max(2, int(seconds / max(per_it, 1e-6)))
        t = time.perf_counter()
        sol = O.solve(mask, mat, P.path[:1], max_iter=n_it)
        dt = time.perf_counter() - t
        return int(sol.records["iterations"].sum()), dt

    cores = O.threads()
    its, dt = timed(budget_s)
    O.set_threads(1)
    try:
        its1, dt1 = timed(single_s)
    finally:
        O.set_threads(cores)
    return {"value": P.L * P.L * its / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first increment of {P.name}, {its} iterations ({dt:.1f} s, OpenMP over {cores} threads)",
            "single_thread": {"value": P.L * P.L * its1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"first increment of {P.name}, {its1} iterations ({dt1:.1f} s)"},
            "host": {"cpu": host_cpu(), "nproc": os.cpu_count()}}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle as O
    probs, cfg = workload(args.workload, args.cap)
    P = probs[0]
    mask = O.mask(P.L, P.f, P.seed)
    mat = O.material()
    O.build()
    t = time.perf_counter()
    O.solve(mask, mat, P.path[:1], max_iter=2)
    per_it = (time.perf_counter() - t) / 2
    # iterations per step: a bounded sample of one increment (~20 s for the whole run)
    n_it = max(2, int(20.0 / max(per_it, 1e-6) / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        O.solve(mask, mat, P.path[:1], max_iter=n_it)
    times = []
    its = 0
    for _ in range(args.steps):
        t = time.perf_counter()
        sol = O.solve(mask, mat, P.path[:1], max_iter=n_it)
        times.append(time.perf_counter() - t)
        its += int(sol.records["iterations"].sum())
    tot = sum(times)
    v = P.L * P.L * its / tot
    cores = O.threads()
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n_it} iterations of the first increment of {P.name} per step",
                         "host": {"cpu": host_cpu(), "nproc": os.cpu_count()}},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


def timed_solves(B, ctx, stream, flush, probs, paths, steps, torch):
    """`steps` batch solves, each bracketed by CUDA events on the context
    stream after an L2 flush; returns (seconds, pixel-iterations, launches,
    last records)."""
    ev = []
    pix_its = 0
    launches = 0
    recs = None
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
        rc, recs = B.epfft_solve_batch(ctx, probs, paths)
        with torch.cuda.stream(stream):
            b.record(stream)
        ev.append((a, b))
        pix_its += sum(p.L * p.L * int(r["iterations"].sum()) for p, r in zip(probs, recs))
        launches += B.epfft_last_stats(ctx)["kernel_launches"]
    stream.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / 1e3, pix_its, launches, recs


def refined_vs_plain(B, ctx, stream, flush, mask, L, path, torch, tol=1e-8, tol_switch=0.0, cap=60000):
    """Solves/s at one equilibrium tolerance that the FP32 path cannot
    certify alone: the plain FP64 solve against the mixed-precision solve
    (FP32 iterations to tol_switch, then FP64 to tol) and against the
    defect-correction form (FP64 state, FP32 transforms of p - p_ref), on the
    increments of `path`; one L2-flushed, CUDA-event-timed solve of each
    after a warm-up."""
    import dataclasses
    prob = B.Problem(L=L, precision="fp64", mask=mask, tol_eq=tol, tol_macro=tol, max_iter=cap)
    warm = B.Problem(L=L, precision="fp64", mask=mask, tol_eq=tol, tol_macro=tol, max_iter=20)
    dprob = dataclasses.replace(prob, precision="fp32_defect")
    B.epfft_autotune(ctx, L, "fp32")
    B.epfft_autotune(ctx, L, "fp32_defect")
    B.epfft_solve(ctx, warm, path[:1])
    B.epfft_solve_refined(ctx, warm, path[:1], tol_switch)
    B.epfft_solve(ctx, dataclasses.replace(warm, precision="fp32_defect"), path[:1])

    def timed(fn):
        with torch.cuda.stream(stream):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
        r = fn()
        with torch.cuda.stream(stream):
            b.record(stream)
        stream.synchronize()
        return a.elapsed_time(b) / 1e3, r

    t64, (rc64, r64) = timed(lambda: B.epfft_solve(ctx, prob, path))
    tr, (rcr, rr, rr32) = timed(lambda: B.epfft_solve_refined(ctx, prob, path, tol_switch))
    td, (rcd, rd) = timed(lambda: B.epfft_solve(ctx, dprob, path))
    return {"workload": f"first {len(path)} increments of the same lattice and path, tol {tol:g} (eta1, eta2) "
                        f"certified in FP64, at most {cap} iterations per increment",
            "fp64_plain": {"solves_per_s": 1.0 / t64, "iterations": int(r64["iterations"].sum()),
                           "converged": bool((r64["status"] == 0).all())},
            "fp32_then_fp64": {"solves_per_s": 1.0 / tr, "tol_switch": tol_switch,
                               "iterations_fp32": int(rr32["iterations"].sum()),
                               "iterations_fp64": int(rr["iterations"].sum()),
                               "converged": bool((rr["status"] == 0).all()),
                               "max_eta1": float(rr["eta1"].max()),
                               "fp32_stage_reached": {"eta1": rr32["eta1"].tolist(), "eta2": rr32["eta2"].tolist(),
                                                      "status": rr32["status"].tolist()}},
            "fp32_defect": {"solves_per_s": 1.0 / td, "iterations": int(rd["iterations"].sum()),
                            "converged": bool((rd["status"] == 0).all()), "max_eta1": float(rd["eta1"].max()),
                            "max_eta2": float(rd["eta2"].max()), "refresh_steps": DEFECT_REFRESH},
            "speedup": t64 / tr, "speedup_defect": t64 / td}


# iterations between refreshes of the defect form's FP64 reference (the
# library's default)
DEFECT_REFRESH = 256


def batched_at_tol(B, ctx, stream, flush, torch, tol=1e-8, cap=60000):
    """The batched forms at one equilibrium tolerance: 8 lattices of the
    batched workload's recipe (L = 512; f = 0.05 and 0.10, seeds 0, 1
    equibiaxial to 2x and 8, 9 shear to 3x the void-free yield strain), the
    first of their 30 increments, tol 1e-8, advanced together in one call:
    plain FP64 against the defect-correction form.  One L2-flushed,
    CUDA-event-timed call of each after a warm-up.  The plain FP32 form
    cannot reach the tolerance (its transforms stall near eta1 ~ 1e-6)."""
    from paper_0802_2488_gb300 import inputs
    lat = [(f, s) for f in (0.05, 0.10) for s in (0, 1, 8, 9)]
    paths = [inputs.load_path("equibiaxial" if s < 8 else "shear", 30, 2.0 if s < 8 else 3.0)[:1] for f, s in lat]

    def probs(prec, it):
        return [B.Problem(L=512, precision=prec, void_fraction=f, seed=s, tol_eq=tol, tol_macro=tol, max_iter=it)
                for f, s in lat]
    out = {"workload": f"{len(lat)} lattices of L=512 (f in {{0.05, 0.10}}, seeds 0, 1 equibiaxial to 2x yield "
                       f"and 8, 9 shear to 3x yield, first of 30 increments), tol {tol:g} (eta1, eta2), at most "
                       f"{cap} iterations; one batched call per form (CUDA events), and the same lattices "
                       f"submitted together to the serving engine (host clock)"}
    for prec in ("fp64", "fp32_defect"):
        B.epfft_autotune(ctx, 512, prec, n_batch=len(lat))
        B.epfft_solve_batch(ctx, probs(prec, 20), paths)
        with torch.cuda.stream(stream):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
        rc, recs = B.epfft_solve_batch(ctx, probs(prec, cap), paths)
        with torch.cuda.stream(stream):
            b.record(stream)
        stream.synchronize()
        t = a.elapsed_time(b) / 1e3
        its = [int(r["iterations"].sum()) for r in recs]
        conv = all(bool((r["status"] == 0).all()) for r in recs)
        out[prec] = {"s": t, "solves_per_s": len(lat) / t, "solves_per_s_at_tol": len(lat) / t if conv else None,
                     "converged": sum(int((r["status"] == 0).all()) for r in recs), "iterations": its,
                     "pixel_iterations_per_s": 512 * 512 * sum(its) / t,
                     "max_eta1": max(float(r["eta1"].max()) for r in recs)}
    out["speedup_defect"] = out["fp64"]["s"] / out["fp32_defect"]["s"]
    # the same lattices through the serving engine (all submitted at once,
    # advanced by serve steps until every ticket is done; host clock)
    for prec in ("fp64", "fp32_defect"):
        B.epfft_serve_open(ctx, 64 << 30, len(lat), 256)
        try:
            t0 = time.perf_counter()
            ps = probs(prec, cap)
            tickets = [B.epfft_submit(ctx, p, q) for p, q in zip(ps, paths)]
            res = [None] * len(lat)
            while any(r is None for r in res):
                B.epfft_serve_step(ctx)
                for i, t in enumerate(tickets):
                    if res[i] is None:
                        res[i] = B.epfft_poll(ctx, t, ps[i], 1)
            t = time.perf_counter() - t0
        finally:
            B.epfft_serve_close(ctx)
        conv = all(r[0] == B.EPFFT_OK for r in res)
        out[f"served_{prec}"] = {"s": t, "solves_per_s": len(lat) / t,
                                 "solves_per_s_at_tol": len(lat) / t if conv else None,
                                 "iterations": [int(r[1]["iterations"].sum()) for r in res],
                                 "p50_latency_s": float(np.percentile([r[3] for r in res], 50)),
                                 "p99_latency_s": float(np.percentile([r[3] for r in res], 99))}
    out["served_speedup_defect"] = out["served_fp64"]["s"] / out["served_fp32_defect"]["s"]
    return out


def convergence(recs, tol: float = 1e-8) -> dict:
    """What the increments of a step reached: how many met both tolerances
    before the cap (status 0), how many stopped at the cap (status 1), and
    eta1 / eta2 at the accepted iterate."""
    st = np.concatenate([np.asarray(r["status"]) for r in recs])
    e1 = np.concatenate([np.asarray(r["eta1"]) for r in recs])
    e2 = np.concatenate([np.asarray(r["eta2"]) for r in recs])
    its = np.concatenate([np.asarray(r["iterations"]) for r in recs])
    return {"tol": tol, "increments": int(st.size), "converged": int((st == 0).sum()),
            "capped": int((st == 1).sum()), "numeric_failures": int((st == 2).sum()),
            "eta1_max": float(e1.max()), "eta1_median": float(np.median(e1)),
            "eta2_max": float(e2.max()), "eta2_median": float(np.median(e2)),
            "iterations_per_increment_mean": float(its.mean())}


def peaks(B, ctx, precision):
    """Roofline denominators: the measured HBM copy rate (MEASURED_PEAKS.json)
    for the FP32 passes; the FP64 FMA rate measured here on this device
    (epfft_fp64_peak) for the FP64 passes."""
    if precision in ("fp32", "fp32_defect"):
        mp = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(mp):
            return json.load(open(mp))["hbm_gbs"], "MEASURED_PEAKS.json hbm_gbs (of measured)"
        return 6800.0, "fallback 6800 GB/s (of fallback)"
    r = B.epfft_fp64_peak(ctx)
    return r["tflops"], (f"measured here: FP64 FMA chains on all {r['n_sm']} SMs, CUDA events, best of 5 "
                         f"({r['ms']:.3f} ms per launch) (of measured)")


def pass_kernels(precision, L, tiling):
    """Names of the two compiled passes a solve of this size runs."""
    rt = "double" if precision == "fp64" else "float"
    if precision == "fp32_defect":
        col = f"col_pass_rs<{L}>" if (tiling == 0 and L >= 128) else f"col_pass<float,{L},{tiling}>"
        return {"row": f"row_pass_dc<{L},{tiling}>", "col": col}
    if precision == "fp32" and tiling == 2:
        return {"row": f"row_pass_rs<{L}>", "col": f"col_pass_rs<{L}> (digit-reversed rows)"}
    col = f"col_pass_rs<{L}>" if (precision == "fp32" and tiling == 0 and L >= 128) else f"col_pass<{rt},{L},{tiling}>"
    return {"row": f"row_pass<{rt},{L},{tiling}>", "col": col}


# DRAM bytes (read + write) per launch from ncu launch lists of the same
# kernels at the same launch shape: (precision, L, solves, tiling, pass) ->
# (bytes, summary under profiles/, digest of the kernel headers the capture
# ran, kernel_source_digest).  An entry whose headers changed since reads
# null until the capture is taken again.
TRAFFIC = {
    ("fp32", 512, 64, 0, "row"): (1211.3e6, "profiles/passes_fp32_c3_c4_launches.md", "4e717a09d0dd1e39"),
    ("fp32", 512, 64, 0, "col"): (354.1e6, "profiles/passes_fp32_c3_c4_launches.md", "4e717a09d0dd1e39"),
    ("fp32", 4096, 1, 2, "row"): (1247.5e6, "profiles/passes_fp32_c3_c4_launches.md", "4e717a09d0dd1e39"),
    ("fp32", 4096, 1, 2, "col"): (358.4e6, "profiles/passes_fp32_c3_c4_launches.md", "4e717a09d0dd1e39"),
    ("fp32_defect", 512, 64, 0, "row"): (2075.0e6, "profiles/defect_passes_c3.md", "c502f6a61a2f68ef"),
    ("fp32_defect", 512, 64, 0, "col"): (353.8e6, "profiles/defect_passes_c3.md", "c502f6a61a2f68ef"),
}


# the kernel headers the passes of each form compile from
PASS_HEADERS = ["common.cuh", "fft.cuh", "tables.cuh", "physics.cuh", "passes.cuh", "colrs.cuh", "rowrs.cuh"]
DEFECT_HEADERS = PASS_HEADERS + ["dcpass.cuh"]


def kernel_source_digest(headers=None):
    """sha256 (first 16 hex digits) over the names and bytes of the kernel
    headers a form's passes compile from (default: those of the FP32 and
    FP64 passes), in name order."""
    import hashlib
    h = hashlib.sha256()
    for name in sorted(headers or PASS_HEADERS):
        h.update(name.encode())
        with open(os.path.join(ROOT, "paper_0802_2488_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_of(precision, L, nb, tiling, k):
    tr = TRAFFIC.get((precision, L, nb, tiling, k))
    if tr is None:
        return None
    heads = DEFECT_HEADERS if precision == "fp32_defect" else PASS_HEADERS
    return tr if kernel_source_digest(heads) == tr[2] else None


def roofline(precision, L, nb, col_ms, row_ms, peak, peak_source, tiling=None):
    """Both fused passes against their roof, from this run's CUDA-event pass
    timings; the dominant (longer) pass is the line's `roofline`.
    FP32 (HBM): algorithmic bytes per pixel, row pass 73 (spectrum read and
    written 24, sigma of iterate n read 16, new strain and sigma written 32,
    void mask 1), column pass 24 (spectrum read and written).
    Defect form (HBM): row pass 113 (spectrum 24, the stress difference of
    iterate n read 16, the new strain and stress differences written 32, the
    reference data read 40, mask 1), column pass 24.
    FP64 (FP64 ALU): flops per pixel, row pass 15 log2 L + 60 (row
    transforms, local step), column pass 15 log2 L + 25 (column transforms,
    Green operator)."""
    n = L * L * nb
    lg = int(np.log2(L))
    if precision in ("fp32", "fp32_defect"):
        work = {"row": (73 if precision == "fp32" else 113) * n, "col": 24 * n}
        unit, scale, bound = "GB/s", 1e9, "hbm"
    else:
        work = {"row": (15 * lg + 60) * n, "col": (15 * lg + 25) * n}
        unit, scale, bound = "TFLOP/s", 1e12, "alu"
    ms = {"row": row_ms, "col": col_ms}
    names = pass_kernels(precision, L, tiling)
    passes = {}
    for k in ("row", "col"):
        a = work[k] / (ms[k] * 1e-3) / scale
        tr = traffic_of(precision, L, nb, tiling, k)
        passes[k] = {"kernel": names[k], "ms": ms[k], "achieved": a, "frac": a / peak,
                     "work_per_launch": work[k], "traffic": tr[0] if tr else None}
    dom = "row" if row_ms >= col_ms else "col"
    d = passes[dom]
    tr = traffic_of(precision, L, nb, tiling, dom)
    if tr:
        note = (f"DRAM read + write per launch from the ncu launch list in {tr[1]} (same kernel headers, "
                f"digest {tr[2]}, and launch shape)")
    elif (precision, L, nb, tiling, dom) in TRAFFIC:
        note = "null: the kernel headers changed since the ncu capture"
    else:
        note = "null: no ncu capture of this kernel at this launch shape"
    return {"bound": bound, "kernel": d["kernel"], "achieved": d["achieved"], "peak": peak, "unit": unit,
            "frac": d["frac"], "traffic": tr[0] if tr else None, "traffic_note": note,
            "peak_source": peak_source, "passes": passes,
            "timing": "epfft_time_passes: CUDA events around each launch on the context stream, mean of the "
                      "timed launches, the same launch shape as the solve"}


def solve_line(B, ctx, stream, flush, torch, name, precision, cap, steps, warmup, e2e_steps, local, ws,
               peak, peak_source, barrier):
    """One batched-solve workload: device-timed steps (inputs in HBM, L2
    flushed between steps), the end-to-end steps with host buffers, the pass
    timings and the convergence reached.  Returns the pieces of a line."""
    probs, cfg = workload(name, cap)
    L = probs[0].L
    nb = len(probs)
    masks_dev = [B.epfft_mask(P.L, P.f, P.seed, device=local) for P in probs]
    masks_host = []
    for m in masks_dev:
        h = torch.empty((L, L), dtype=torch.uint8, pin_memory=True)
        h.copy_(m.cpu())
        masks_host.append(h.numpy())
    paths = [P.path for P in probs]

    def problems(host):
        return [B.Problem(L=L, precision=precision, mask=(masks_host[i] if host else masks_dev[i]), tol_eq=1e-8,
                          tol_macro=1e-8, max_iter=cap) for i in range(nb)]

    # the autotuner picks the tiling of this lattice size (outside the timed region)
    tiling, tiling_ms = B.epfft_autotune(ctx, L, precision, n_batch=nb)
    cfg["tiling"] = {"chosen": tiling, "ms_per_iteration": tiling_ms}
    pd = problems(False)
    for _ in range(warmup):
        B.epfft_solve_batch(ctx, pd, paths)
    barrier()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        dev_s, pix_its, launches, recs = timed_solves(B, ctx, stream, flush, pd, paths, steps, torch)
        barrier()
        wall = time.perf_counter() - t0
    clocks = clk.summary()

    # end to end through the C ABI with host buffers (pinned masks in; records,
    # final strain, plastic flags and cluster labels out into pinned buffers
    # the caller allocates once and reuses)
    ph = problems(True)
    outs = [B.pinned_fields(P, len(path)) for P, path in zip(ph, paths)]
    B.epfft_solve_batch(ctx, ph, paths, fields=True, out=outs)
    barrier()
    t0 = time.perf_counter()
    e2e_its = 0
    for _ in range(e2e_steps):
        rc, rr, ff = B.epfft_solve_batch(ctx, ph, paths, fields=True, out=outs)
        e2e_its += sum(p.L * p.L * int(r["iterations"].sum()) for p, r in zip(ph, rr))
    barrier()
    e2e_s = time.perf_counter() - t0
    rs = 4 if precision == "fp32" else 8  # the defect form's fields are FP64
    h2d = sum(L * L + 4 * 8 * P.n_inc for P in probs)
    d2h = sum(P.n_inc * 104 + L * L * 4 * rs + P.n_inc * L * L * 5 for P in probs)

    # pass timing (CUDA events on the context stream) for the roofline
    E_mid = probs[0].path[probs[0].n_inc // 2]
    n_pass = 20 if L * L * nb >= (1 << 24) else 50
    col_ms, row_ms = B.epfft_time_passes(ctx, pd[0], E_mid, n_pass, n_batch=nb)

    t_step = dev_s / steps
    t_step, dev_s, e2e_s = max_over_ranks([t_step, dev_s, e2e_s], device=torch.device(f"cuda:{local}"))
    conv = convergence(recs)
    sps = job_value(ws, steps * nb, dev_s)
    cfg.update(l2="inputs larger than L2 at this size; L2 also flushed between steps (512 MiB write, outside "
                  "the step events)" if L * L * nb >= (1 << 22) else
               "flushed between steps (512 MiB write, outside the step events)",
               parallelism="replicas" if ws > 1 else "single GPU", precision=precision,
               solves_per_s=sps, solves_per_s_at_tol=sps if conv["converged"] == conv["increments"] else None)
    return {
        "value": job_value(ws, pix_its, dev_s), "ms_per_step": 1e3 * t_step, "config": cfg,
        "convergence": conv,
        "roofline": roofline(precision, L, nb, col_ms, row_ms, peak, peak_source, tiling),
        "e2e": {"value": job_value(ws, e2e_its, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps},
        "gpu_launches": launches, "clocks": clocks, "wall_s": wall, "recs": recs, "probs": probs,
        "masks_dev": masks_dev,
    }


def serving(B, ctx, local, ws, rank, precision="fp32", cap=20, n_requests=150):
    """C5: Poisson request stream through the serving engine; latency =
    completion - arrival on the host clock."""
    from paper_0802_2488_gb300 import inputs

    def prob(r):
        P = r.problem
        return B.Problem(L=P.L, precision=precision, void_fraction=P.f, seed=P.seed, tol_eq=1e-8,
                         tol_macro=1e-8, max_iter=cap)

    # tilings of the served sizes: single solves (the solo probe) and the
    # 16-slot serving classes
    for L in (128, 256, 512, 1024):
        B.epfft_autotune(ctx, L, precision, n_batch=1)
        B.epfft_autotune(ctx, L, precision, n_batch=16)
    # solo capacity: a few requests run back to back, one at a time
    probe = inputs.serving_stream(12, 1.0, seed=1000 + rank)
    for r in probe[:2]:
        B.epfft_solve(ctx, prob(r), r.problem.path)
    t0 = time.perf_counter()
    for r in probe[2:]:
        B.epfft_solve(ctx, prob(r), r.problem.path)
    solo = (len(probe) - 2) / (time.perf_counter() - t0)
    rate = 0.7 * solo
    reqs = inputs.serving_stream(n_requests, rate, seed=rank)
    budget = 16 << 30
    B.epfft_serve_open(ctx, budget, 16, 32)
    lat, pix = [], 0
    launches = 0
    recs = []
    h2d = d2h = 0  # strain paths submitted, records read back (masks are generated on the device)
    tickets = {}
    nxt = 0
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        while nxt < len(reqs) or tickets:
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt].arrival_s <= now:
                r = reqs[nxt]
                tickets[nxt] = (B.epfft_submit(ctx, prob(r), r.problem.path), r)
                h2d += r.problem.path.size * 8
                nxt += 1
            if not tickets:
                time.sleep(max(0.0, min(0.01, reqs[nxt].arrival_s - now)))
                continue
            B.epfft_serve_step(ctx)
            launches += B.epfft_last_stats(ctx)["kernel_launches"]
            done_t = time.perf_counter() - t0
            for i, (t, r) in list(tickets.items()):
                res = B.epfft_poll(ctx, t, prob(r), r.problem.n_inc)
                if res is not None:
                    lat.append(done_t - r.arrival_s)
                    pix += r.problem.L ** 2 * int(res[1]["iterations"].sum())
                    recs.append(res[1])
                    d2h += res[1].nbytes
                    del tickets[i]
        total = time.perf_counter() - t0
    B.epfft_serve_close(ctx)
    clocks = clk.summary()
    lat = np.array(lat)
    conv = convergence(recs)
    return {
        "value": ws * pix / total, "unit": UNIT, "ms_per_step": 1e3 * total,
        "workload": f"Poisson stream of {len(reqs)} requests at {rate:.2f}/s (70% of the measured solo capacity "
                    f"{solo:.2f}/s): L uniform in {{128,256,512,1024}}, f uniform in [0.05,0.35], equibiaxial or "
                    f"shear, 10-50 increments, seed = request id; FP32 fields, FP64 reductions; at most {cap} "
                    f"iterations per increment; HBM budget 16 GiB, 16 slots per size",
        "rate_per_s": rate, "solo_capacity_per_s": solo,
        "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
        "solves_per_s": len(lat) / total,
        "solves_per_s_at_tol": len(lat) / total if conv["converged"] == conv["increments"] else None,
        "convergence": conv,
        # timed on the host clock from the first arrival to the last result,
        # through submit / serve_step / poll: value and e2e are the same
        # end-to-end measurement
        "e2e": {"value": ws * pix / total, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches, "clocks": clocks,
    }


def fp32_vs_fp64(B, ctx, stream, flush, torch, steps, warmup, local, barrier, peak64, src64):
    """C2 (L = 256, shear): plain FP64 solve, its FP32 form at the same
    iteration cap with the errors of the final strain field, the plastic
    flags and the macroscopic curve against FP64, and plain FP64 against the
    mixed-precision solve at a tolerance both reach."""
    out = {}
    line64 = solve_line(B, ctx, stream, flush, torch, "c2", "fp64", CAPS["c2"], steps, warmup, 1, local, 1,
                        peak64, src64, barrier)
    hbm, hsrc = peaks(B, ctx, "fp32")
    line32 = solve_line(B, ctx, stream, flush, torch, "c2", "fp32", CAPS["c2"], steps, warmup, 1, local, 1,
                        hbm, hsrc, barrier)
    for key, ln in (("fp64", line64), ("fp32", line32)):
        out[key] = {k: ln[k] for k in ("value", "ms_per_step", "convergence", "roofline", "e2e", "clocks")}
        out[key]["solves_per_s"] = ln["config"]["solves_per_s"]
        out[key]["solves_per_s_at_tol"] = ln["config"]["solves_per_s_at_tol"]
        out[key]["tiling"] = ln["config"]["tiling"]
    out["workload"] = line64["config"]["workload"]
    # final fields of both precisions at the same cap (one untimed solve each)
    P = line64["probs"][0]
    mask = line64["masks_dev"][0]
    f = {}
    for prec in ("fp64", "fp32"):
        pr = B.Problem(L=P.L, precision=prec, mask=mask, tol_eq=1e-8, tol_macro=1e-8, max_iter=CAPS["c2"])
        rc, rec, fl = B.epfft_solve(ctx, pr, P.path, fields=True)
        f[prec] = (rec, fl)
    (r64, f64), (r32, f32) = f["fp64"], f["fp32"]
    e64, e32 = f64.eps.astype(np.float64), f32.eps.astype(np.float64)
    s64, s32 = r64["sig_mean"], r32["sig_mean"]
    out["fp32_errors_vs_fp64"] = {
        "same_iterations": bool(np.array_equal(r64["iterations"], r32["iterations"])),
        "final_strain_rel_l2": float(np.linalg.norm(e32 - e64) / np.linalg.norm(e64)),
        "macro_stress_curve_max_rel_err": float(np.max(np.linalg.norm(s32 - s64, axis=1) /
                                                       np.linalg.norm(s64, axis=1))),
        "macro_strain_curve_max_rel_err": float(np.max(np.linalg.norm(r32["eps_mean"] - r64["eps_mean"], axis=1) /
                                                       np.linalg.norm(r64["eps_mean"], axis=1))),
        "plastic_flag_disagreements_per_increment_max": int(np.max(np.sum(f32.plastic != f64.plastic,
                                                                          axis=(1, 2)))),
        "eta1_fp32_last_increment": float(r32["eta1"][-1]), "eta1_fp64_last_increment": float(r64["eta1"][-1]),
        "note": "both solves stop at the same iteration cap per increment (neither converges to 1e-8 on most "
                "increments), so this is the FP32 rounding effect on the same iterates",
    }
    out["refined"] = refined_vs_plain(B, ctx, stream, flush, mask, P.L, P.path[:2], torch)
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    from paper_0802_2488_gb300 import binding as B
    from paper_0802_2488_gb300 import build
    build.build()
    stream = torch.cuda.Stream(device=local)
    ctx = B.Context(local, stream=stream.cuda_stream)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(local)

    if args.workload == "c5":
        r = serving(B, ctx, local, ws, rank, args.precision, args.cap, args.requests)
        if rank == 0:
            out = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": 1, "warmup": 0,
                   "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                   "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
                   "config": {"workload": r["workload"], "precision": args.precision, "parallelism": "single GPU",
                              "rate_per_s": r["rate_per_s"], "latency_p50_s": r["latency_p50_s"],
                              "latency_p99_s": r["latency_p99_s"], "solves_per_s": r["solves_per_s"],
                              "solves_per_s_at_tol": r["solves_per_s_at_tol"],
                              "l2": "inputs of the running set exceed L2 at the larger sizes; not flushed"},
                   "convergence": r["convergence"], "e2e": r["e2e"], "gpu_launches": r["gpu_launches"],
                   "clocks": r["clocks"]}
            print(json.dumps(out), flush=True)
        ctx.close()
        return

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=local)
    peak, peak_src = peaks(B, ctx, args.precision)
    line = solve_line(B, ctx, stream, flush, torch, args.workload, args.precision, args.cap, args.steps,
                      args.warmup, min(args.steps, 5), local, ws, peak, peak_src, barrier)
    extras = {}
    default_run = args.workload == "c3" and args.precision == "fp32" and args.cap == CAPS["c3"]
    if default_run and ws == 1 and not args.no_extras:
        # the other configurations, measured in the same process (shorter
        # step counts: each is a sub-object, not the headline)
        c4 = solve_line(B, ctx, stream, flush, torch, "c4", "fp32", CAPS["c4"], 2, 1, 1, local, ws, peak,
                        peak_src, barrier)
        extras["c4"] = {k: c4[k] for k in ("value", "ms_per_step", "convergence", "roofline", "e2e", "clocks",
                                           "gpu_launches")}
        extras["c4"]["config"] = {k: v for k, v in c4["config"].items()}
        extras["c4"]["steps"], extras["c4"]["warmup"] = 2, 1
        extras["c5"] = serving(B, ctx, local, ws, rank, "fp32", CAPS["c5"], args.requests)
        p64, s64 = peaks(B, ctx, "fp64")
        extras["c2"] = fp32_vs_fp64(B, ctx, stream, flush, torch, min(args.steps, 3), 1, local, barrier, p64, s64)
        extras["c2"]["steps"], extras["c2"]["warmup"] = min(args.steps, 3), 1
        extras["batched_at_tol"] = batched_at_tol(B, ctx, stream, flush, torch)
        # the batched workload in the defect form (same cap): its throughput and
        # the roofline of its passes
        c3d = solve_line(B, ctx, stream, flush, torch, "c3", "fp32_defect", CAPS["c3"], 2, 1, 1, local, ws, peak,
                         peak_src, barrier)
        extras["c3_defect"] = {k: c3d[k] for k in ("value", "ms_per_step", "convergence", "roofline", "e2e",
                                                    "clocks", "gpu_launches")}
        extras["c3_defect"]["config"] = c3d["config"]
        extras["c3_defect"]["steps"], extras["c3_defect"]["warmup"] = 2, 1

    if rank == 0:
        out = {
            "metric": METRIC, "value": line["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": line["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
            "data": "synthetic", "config": line["config"], "convergence": line["convergence"],
            "roofline": line["roofline"], "e2e": line["e2e"], "gpu_launches": line["gpu_launches"],
            "clocks": line["clocks"], "wall_s": line["wall_s"],
        }
        out.update(extras)
        if ws == 1 and not args.no_baseline:
            out["cpu_baseline"] = cpu_baseline(line["probs"])
        print(json.dumps(out), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
