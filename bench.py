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
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--cap", type=int, default=1000, help="max iterations per increment")
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU-baseline leg")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(cap: int):
    from paper_0802_2488_gb300 import inputs
    P = inputs.config2()
    return P, dict(workload=f"{P.name}: L=256, f=0.20 Bernoulli voids (seed 0), shear E12 to 3x yield "
                            f"in 40 increments, mu=1 lambda=1.5 Y=1, C0=matrix, tol 1e-8 (eta1, eta2), "
                            f"max {cap} iterations per increment, clusters labelled per increment",
                   L=P.L, void_fraction=P.f, seed=P.seed, loading=P.mode, n_inc=P.n_inc,
                   max_iter_per_increment=cap, tol=1e-8)


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


def cpu_baseline(cap: int, budget_s: float = 15.0):
    """The oracle as it stands, on this machine's host cores (OpenMP), on a
    bounded sample of the workload: the first increment of the shear path
    on the same lattice, with as many iterations as fit in ~budget_s."""
    import oracle as O
    from paper_0802_2488_gb300 import inputs
    P = inputs.config2()
    mask = O.mask(P.L, P.f, P.seed)
    mat = O.material()
    O.build()
    t = time.perf_counter()
    O.solve(mask, mat, P.path[:1], max_iter=3)
    per_it = (time.perf_counter() - t) / 3
    n_it = max(3, min(cap, int(budget_s / max(per_it, 1e-6))))
    t = time.perf_counter()
    sol = O.solve(mask, mat, P.path[:1], max_iter=n_it)
    dt = time.perf_counter() - t
    its = int(sol.records["iterations"].sum())
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": P.L * P.L * its / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first increment of the L=256 shear workload, {its} iterations "
                      f"({dt:.1f} s, OpenMP over {cores} threads)"}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle as O
    from paper_0802_2488_gb300 import inputs
    P, cfg = workload(args.cap)
    mask = O.mask(P.L, P.f, P.seed)
    mat = O.material()
    O.build()
    n_it = 20  # iterations per step: a bounded sample of one increment
    for _ in range(args.warmup):
        O.solve(mask, mat, P.path[:1], max_iter=2)
    times = []
    its = 0
    for _ in range(args.steps):
        t = time.perf_counter()
        sol = O.solve(mask, mat, P.path[:1], max_iter=n_it)
        times.append(time.perf_counter() - t)
        its += int(sol.records["iterations"].sum())
    tot = sum(times)
    v = P.L * P.L * its / tot
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n_it} iterations of the first increment per step"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


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
    P, cfg = workload(args.cap)
    stream = torch.cuda.Stream(device=local)
    ctx = B.Context(local, stream=stream.cuda_stream)
    mask_dev = B.epfft_mask(P.L, P.f, P.seed, device=local)
    mask_host = torch.empty((P.L, P.L), dtype=torch.uint8, pin_memory=True)
    mask_host.copy_(mask_dev.cpu())
    mask_host_np = mask_host.numpy()
    prob_dev = B.Problem(L=P.L, precision=args.precision, mask=mask_dev, tol_eq=1e-8, tol_macro=1e-8,
                         max_iter=args.cap)
    prob_host = B.Problem(L=P.L, precision=args.precision, mask=mask_host_np, tol_eq=1e-8, tol_macro=1e-8,
                          max_iter=args.cap)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=local)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(local)

    # warm-up
    for _ in range(args.warmup):
        B.epfft_solve(ctx, prob_dev, P.path)

    # timed region (device): inputs resident in HBM
    pix_its = 0
    launches = 0
    ev = []
    barrier()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
            rc, rec = B.epfft_solve(ctx, prob_dev, P.path)
            with torch.cuda.stream(stream):
                b.record(stream)
            ev.append((a, b))
            pix_its += P.L * P.L * int(rec["iterations"].sum())
            launches += B.epfft_last_stats(ctx)["kernel_launches"]
        barrier()
        wall = time.perf_counter() - t0
    dev_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    clocks = clk.summary()

    # end to end through the C ABI with host buffers
    for _ in range(1):
        B.epfft_solve(ctx, prob_host, P.path, fields=True)
    barrier()
    t0 = time.perf_counter()
    e2e_its = 0
    for _ in range(args.steps):
        rc, rec, f = B.epfft_solve(ctx, prob_host, P.path, fields=True)
        e2e_its += P.L * P.L * int(rec["iterations"].sum())
    barrier()
    e2e_s = time.perf_counter() - t0
    rs = 8 if args.precision == "fp64" else 4
    h2d = P.L * P.L + 4 * 8 * P.n_inc
    d2h = P.n_inc * 104 + P.L * P.L * 4 * rs + 2 * P.n_inc * P.L * P.L * 5

    # pass timing (CUDA events on the context stream) for the roofline
    E_mid = P.path[P.n_inc // 2]
    col_ms, row_ms = B.epfft_time_passes(ctx, prob_dev, E_mid, 200)

    t_step = dev_s / args.steps
    if ws > 1:
        import torch.distributed as dist
        tt = torch.tensor([t_step, dev_s, e2e_s], dtype=torch.float64, device=local)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_step, dev_s, e2e_s = tt.tolist()
    value = ws * pix_its / dev_s
    if rank == 0:
        L = P.L
        lg = int(np.log2(L))
        if args.precision == "fp64":
            # FP64 arithmetic bound: row pass 15 log2 L + 60 flops per pixel
            # (row transforms, local step); column pass 15 log2 L + 25 (column
            # transforms, Green operator)
            row_flops = (15 * lg + 60) * L * L
            col_flops = (15 * lg + 25) * L * L
            dom_ms, dom_flops, dom = (row_ms, row_flops, "row") if row_ms >= col_ms else (col_ms, col_flops, "col")
            sm = clocks.get("sm_max_mhz") or 2070.0
            peak = 152 * 2 * 2 * sm * 1e6 / 1e12  # 152 SMs x 2 FP64 FMA/clk x 2 flop
            achieved = dom_flops / (dom_ms * 1e-3) / 1e12
            roof = {"bound": "alu", "kernel": f"{dom}_pass<double,{L}>", "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                    "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x max SM clock"}
        else:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
                os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
            row_b, col_b = 57 * L * L, 24 * L * L
            dom_ms, dom_b, dom = (row_ms, row_b, "row") if row_ms >= col_ms else (col_ms, col_b, "col")
            achieved = dom_b / (dom_ms * 1e-3) / 1e9
            roof = {"bound": "hbm", "kernel": f"{dom}_pass<float,{L}>", "achieved": achieved,
                    "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                    "traffic": None, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
        roof.update({"col_pass_ms": col_ms, "row_pass_ms": row_ms})
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
            "data": "synthetic",
            "config": dict(cfg, l2="flushed between steps (512 MiB write, outside the step events)",
                           parallelism="replicas" if ws > 1 else "single GPU",
                           solves_per_s=ws * args.steps / dev_s, precision=args.precision),
            "roofline": roof,
            "e2e": {"value": ws * e2e_its / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
            "wall_s": wall,
        }
        if ws == 1 and not args.no_baseline:
            out["cpu_baseline"] = cpu_baseline(args.cap)
        print(json.dumps(out), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
