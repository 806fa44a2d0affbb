#!/usr/bin/env python3
"""Throughput of the augmented-Lagrangian FFT solve (Willot & Pellegrini,
arXiv:0802.2488) on one GB300, printed as one JSON line.

A step is one whole solve of the shear workload: L = 256 lattice, i.i.d.
Bernoulli voids f = 0.20 (seed 0), matrix mu = 1, lambda = 1.5, Y = 1, C0 =
matrix, 40 equal increments of E12 up to 3x the void-free yield strain,
equilibrium and macro tolerances 1e-8, each increment capped at --cap
iterations.  The mask is generated, all increments are iterated, and the
plastic clusters of every increment are labelled.  `value` counts the
pixel-iterations the method needed (sum over increments of L^2 x
iterations) per second of device time with the inputs in HBM; `e2e` is the
same through the C ABI with host buffers (the pinned mask in, records and
the final strain field out) and the copies inside the timed region.
On this workload a single-GPU line also carries the FP32 form of the same
solve (`fp32`) and, at a tolerance both reach (1e-8 on the first
increments), plain FP64 against the mixed-precision solve (`refined`).

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


# DRAM bytes (read + write) per launch of the dominant pass, from one ncu
# capture of the same kernel, tiling and solves per launch
# (profiles/passes_dram_traffic.md); a configuration not listed, or one
# whose kernel changed after the capture, reports null.
TRAFFIC = {
    ("row_pass<double,256>", 1, 1): 3828480,
    ("row_pass<float,512>", 0, 64): 488783104 + 681300480,
    ("row_pass<float,4096>", 0, 1): 542052096 + 696104448,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="epfft", choices=["epfft", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "c5"])
    ap.add_argument("--requests", type=int, default=150, help="c5: requests in the stream")
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32"],
                    help="default: fp64 for c1/c2, fp32 for c3/c4")
    ap.add_argument("--cap", type=int, default=None, help="max iterations per increment")
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-fp32", action="store_true",
                    help="c2: skip the FP32 companion and the mixed-precision comparison "
                         "(both run on single-GPU runs only)")
    a = ap.parse_args()
    if a.precision is None:
        a.precision = "fp64" if a.workload in ("c1", "c2") else "fp32"
    if a.cap is None:
        a.cap = {"c1": 2000, "c2": 300, "c3": 100, "c4": 60, "c5": 20}[a.workload]
    return a


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
    (FP32 iterations to tol_switch, then FP64 to tol), on the increments of
    `path`; one L2-flushed, CUDA-event-timed solve of each after a warm-up."""
    prob = B.Problem(L=L, precision="fp64", mask=mask, tol_eq=tol, tol_macro=tol, max_iter=cap)
    warm = B.Problem(L=L, precision="fp64", mask=mask, tol_eq=tol, tol_macro=tol, max_iter=20)
    B.epfft_autotune(ctx, L, "fp32")
    B.epfft_solve(ctx, warm, path[:1])
    B.epfft_solve_refined(ctx, warm, path[:1], tol_switch)

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
            "speedup": t64 / tr}


def run_serving(args):
    """C5: Poisson request stream through the serving engine."""
    import torch
    from paper_0802_2488_gb300 import binding as B
    from paper_0802_2488_gb300 import build
    from paper_0802_2488_gb300 import inputs
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    ctx = B.Context(local)

    def prob(r):
        P = r.problem
        return B.Problem(L=P.L, precision=args.precision, void_fraction=P.f, seed=P.seed, tol_eq=1e-8,
                         tol_macro=1e-8, max_iter=args.cap)

    # tilings of the served sizes: single solves (the solo probe) and the
    # 16-slot serving classes
    for L in (128, 256, 512, 1024):
        B.epfft_autotune(ctx, L, args.precision, n_batch=1)
        B.epfft_autotune(ctx, L, args.precision, n_batch=16)
    # solo capacity: a few requests run back to back, one at a time
    probe = inputs.serving_stream(12, 1.0, seed=1000 + rank)
    for r in probe[:2]:
        B.epfft_solve(ctx, prob(r), r.problem.path)
    t0 = time.perf_counter()
    for r in probe[2:]:
        B.epfft_solve(ctx, prob(r), r.problem.path)
    solo = (len(probe) - 2) / (time.perf_counter() - t0)
    rate = 0.7 * solo
    reqs = inputs.serving_stream(args.requests, rate, seed=rank)
    budget = 16 << 30
    B.epfft_serve_open(ctx, budget, 16, 32)
    lat, pix = [], 0
    launches = 0
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
                    d2h += res[1].nbytes
                    del tickets[i]
        total = time.perf_counter() - t0
    B.epfft_serve_close(ctx)
    clocks = clk.summary()
    lat = np.array(lat)
    out = {
        "metric": METRIC, "value": ws * pix / total, "unit": UNIT, "n_gpus": ws, "steps": 1, "warmup": 0,
        "ms_per_step": 1e3 * total, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": f"Poisson stream of {len(reqs)} requests at {rate:.2f}/s (70% of the measured "
                               f"solo capacity {solo:.2f}/s): L uniform in {{128,256,512,1024}}, f uniform in "
                               f"[0.05,0.35], equibiaxial or shear, 10-50 increments, seed = request id; at most "
                               f"{args.cap} iterations per increment; HBM budget 16 GiB, 16 slots per size",
                   "rate_per_s": rate, "solo_capacity_per_s": solo,
                   "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                   "solves_per_s": len(lat) / total, "precision": args.precision, "parallelism": "single GPU",
                   "l2": "inputs of the running set exceed L2 at the larger sizes; not flushed"},
        # the stream is timed on the host clock from the first arrival to the
        # last result, through submit / serve_step / poll: value and e2e are
        # the same end-to-end measurement
        "e2e": {"value": ws * pix / total, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches, "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c5":
        return run_serving(args)
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    from paper_0802_2488_gb300 import binding as B
    from paper_0802_2488_gb300 import build
    build.build()
    probs, cfg = workload(args.workload, args.cap)
    L = probs[0].L
    stream = torch.cuda.Stream(device=local)
    ctx = B.Context(local, stream=stream.cuda_stream)
    masks_dev = [B.epfft_mask(P.L, P.f, P.seed, device=local) for P in probs]
    masks_host = []
    for m in masks_dev:
        h = torch.empty((L, L), dtype=torch.uint8, pin_memory=True)
        h.copy_(m.cpu())
        masks_host.append(h.numpy())
    paths = [P.path for P in probs]

    def problems(prec, host):
        return [B.Problem(L=L, precision=prec, mask=(masks_host[i] if host else masks_dev[i]), tol_eq=1e-8,
                          tol_macro=1e-8, max_iter=args.cap) for i in range(len(probs))]

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=local)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(local)

    # the autotuner picks the tiling of this lattice size (outside the timed region)
    tiling, tiling_ms = B.epfft_autotune(ctx, L, args.precision, n_batch=len(probs))
    cfg["tiling"] = {"chosen": tiling, "ms_per_iteration": tiling_ms}
    pd = problems(args.precision, False)
    for _ in range(args.warmup):
        B.epfft_solve_batch(ctx, pd, paths)
    barrier()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        dev_s, pix_its, launches, recs = timed_solves(B, ctx, stream, flush, pd, paths, args.steps, torch)
        barrier()
        wall = time.perf_counter() - t0
    clocks = clk.summary()

    # end to end through the C ABI with host buffers (pinned masks in; records,
    # final strain, plastic flags and cluster labels out into pinned buffers
    # the caller allocates once and reuses)
    ph = problems(args.precision, True)
    outs = [B.pinned_fields(P, len(path)) for P, path in zip(ph, paths)]
    B.epfft_solve_batch(ctx, ph, paths, fields=True, out=outs)
    barrier()
    t0 = time.perf_counter()
    e2e_its = 0
    for _ in range(args.steps):
        rc, rr, ff = B.epfft_solve_batch(ctx, ph, paths, fields=True, out=outs)
        e2e_its += sum(p.L * p.L * int(r["iterations"].sum()) for p, r in zip(ph, rr))
    barrier()
    e2e_s = time.perf_counter() - t0
    rs = 8 if args.precision == "fp64" else 4
    h2d = sum(L * L + 4 * 8 * P.n_inc for P in probs)
    d2h = sum(P.n_inc * 104 + L * L * 4 * rs + P.n_inc * L * L * 5 for P in probs)

    # pass timing (CUDA events on the context stream) for the roofline
    E_mid = probs[0].path[probs[0].n_inc // 2]
    col_ms, row_ms = B.epfft_time_passes(ctx, pd[0], E_mid, 50, n_batch=len(probs))

    companion = None
    if args.workload == "c2" and args.precision == "fp64" and not args.no_fp32 and ws == 1:
        B.epfft_autotune(ctx, L, "fp32")
        pf = problems("fp32", False)
        for _ in range(args.warmup):
            B.epfft_solve_batch(ctx, pf, paths)
        f_s, f_its, _, frecs = timed_solves(B, ctx, stream, flush, pf, paths, args.steps, torch)
        fcol, frow = B.epfft_time_passes(ctx, pf[0], E_mid, 50)
        s64, s32 = recs[0]["sig_mean"], frecs[0]["sig_mean"]
        curve_err = float(np.max(np.linalg.norm(s32 - s64, axis=1) / np.linalg.norm(s64, axis=1)))
        companion = {"value": f_its / f_s, "unit": UNIT, "ms_per_step": 1e3 * f_s / args.steps,
                     "solves_per_s": args.steps / f_s, "col_pass_ms": fcol, "row_pass_ms": frow,
                     "macro_curve_max_rel_err_vs_fp64": curve_err,
                     "eta1_last_increment": float(frecs[0]["eta1"][-1]),
                     "dtype": "f32 fields and FFTs, f64 reductions"}

    refined = None
    if args.workload == "c2" and args.precision == "fp64" and not args.no_fp32 and ws == 1:
        refined = refined_vs_plain(B, ctx, stream, flush, masks_dev[0], L, paths[0][:2], torch)

    t_step = dev_s / args.steps
    t_step, dev_s, e2e_s = max_over_ranks([t_step, dev_s, e2e_s], device=torch.device(f"cuda:{local}"))
    value = job_value(ws, pix_its, dev_s)
    if rank == 0:
        lg = int(np.log2(L))
        nb = len(probs)
        if args.precision == "fp64":
            # FP64 arithmetic bound: row pass 15 log2 L + 60 flops per pixel
            # (row transforms, local step); column pass 15 log2 L + 25 (column
            # transforms, Green operator)
            row_w, col_w = (15 * lg + 60) * L * L * nb, (15 * lg + 25) * L * L * nb
            dom_ms, dom_w, dom = (row_ms, row_w, "row") if row_ms >= col_ms else (col_ms, col_w, "col")
            sm = clocks.get("sm_max_mhz") or 2070.0
            peak = 152 * 2 * 2 * sm * 1e6 / 1e12  # 152 SMs x 2 FP64 FMA/clk x 2 flop
            achieved = dom_w / (dom_ms * 1e-3) / 1e12
            roof = {"bound": "alu", "kernel": f"{dom}_pass<double,{L}>", "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                    "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x max SM clock"}
        else:
            mp = os.path.join(ROOT, "MEASURED_PEAKS.json")
            hbm = json.load(open(mp))["hbm_gbs"] if os.path.exists(mp) else 6800.0
            # row pass: spectrum read + write 24 B, sigma read 16 B, eps and
            # sigma written 32 B, mask 1 B; column pass: spectrum r + w 24 B
            row_b, col_b = 73 * L * L * nb, 24 * L * L * nb
            dom_ms, dom_b, dom = (row_ms, row_b, "row") if row_ms >= col_ms else (col_ms, col_b, "col")
            achieved = dom_b / (dom_ms * 1e-3) / 1e9
            roof = {"bound": "hbm", "kernel": f"{dom}_pass<float,{L}>", "achieved": achieved, "peak": hbm,
                    "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if os.path.exists(mp)
                    else "fallback 6800 GB/s (of fallback)"}
        roof.update({"col_pass_ms": col_ms, "row_pass_ms": row_ms})
        roof["traffic"] = TRAFFIC.get((roof["kernel"], tiling, nb))
        if roof["traffic"] is not None:
            roof["traffic_source"] = "profiles/passes_dram_traffic.md (ncu dram__bytes_read.sum + write.sum per launch)"
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
            "data": "synthetic",
            "config": dict(cfg, l2="flushed between steps (512 MiB write, outside the step events)",
                           parallelism="replicas" if ws > 1 else "single GPU",
                           solves_per_s=job_value(ws, args.steps * len(probs), dev_s), precision=args.precision),
            "roofline": roof,
            "e2e": {"value": job_value(ws, e2e_its, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
            "wall_s": wall,
        }
        if companion:
            out["fp32"] = companion
        if refined:
            out["refined"] = refined
        if ws == 1 and not args.no_baseline:
            out["cpu_baseline"] = cpu_baseline(probs)
        print(json.dumps(out), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
