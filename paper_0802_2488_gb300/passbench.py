"""Time the two fused passes of one iteration for one lattice side and
precision (CUDA events on the context stream, through epfft_time_passes) and
print their algorithmic throughput as JSON.

    python -m paper_0802_2488_gb300.passbench --L 2048 --precision fp32 --iters 50

Algorithmic work per pixel and pass:
  row pass:    bytes 73 (FP32) / 145 (FP64),  flops 15 log2 L + 60
               (spectrum read and written, sigma of iterate n read, the new
               strain and sigma written, the void mask)
  column pass: bytes 24 (FP32) / 48 (FP64),   flops 15 log2 L + 25
"""
from __future__ import annotations

import argparse
import json
import math

from . import binding as B
from . import inputs


def measure(ctx, L: int, precision: str, f: float = 0.2, iters: int = 50, variant: int | None = None,
            batch: int = 1) -> dict:
    if variant is not None:
        B.epfft_set_tiling(ctx, L, precision, variant)
    prob = B.Problem(L=L, precision=precision, void_fraction=f, seed=0)
    E = inputs.load_path("shear", 40, 3.0)[20]
    col_ms, row_ms = B.epfft_time_passes(ctx, prob, E, iters, n_batch=batch)
    n = L * L * batch
    lg = math.log2(L)
    # algorithmic bytes per pixel: FP32 row 73 / column 24, FP64 145 / 48,
    # the defect form 113 (FP32 spectrum, the FP32 differences of iterate n
    # and n+1, the reference data) / 24
    row_b = {"fp64": 145, "fp32": 73, "fp32_defect": 113}[precision] * n
    col_b = (48 if precision == "fp64" else 24) * n
    row_f, col_f = (15 * lg + 60) * n, (15 * lg + 25) * n
    if col_ms == 0.0:
        # the on-chip schedule (tiling 3): one launch, row_ms per iteration
        return {"L": L, "precision": precision, "iters": iters, "variant": variant, "batch": batch,
                "ms_per_iteration": row_ms, "px_it_per_s": n / (row_ms * 1e-3)}
    return {
        "L": L, "precision": precision, "iters": iters, "variant": variant, "batch": batch,
        "col_ms": col_ms, "row_ms": row_ms,
        "col_GBps": col_b / (col_ms * 1e-3) / 1e9, "row_GBps": row_b / (row_ms * 1e-3) / 1e9,
        "col_GFLOPs": col_f / (col_ms * 1e-3) / 1e9, "row_GFLOPs": row_f / (row_ms * 1e-3) / 1e9,
        "px_it_per_s": n / ((col_ms + row_ms) * 1e-3),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, nargs="+", default=[256])
    ap.add_argument("--precision", nargs="+", default=["fp64", "fp32"])
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--batch", type=int, default=1, help="solves per launch")
    ap.add_argument("--variants", type=int, nargs="*", default=None,
                    help="compiled tilings to time (default: the context's choice)")
    a = ap.parse_args()
    from . import build
    build.build()
    with B.Context(0) as ctx:
        for prec in a.precision:
            for L in a.L:
                if B.epfft_supported(L, prec):
                    for v in (a.variants if a.variants else [None]):
                        print(json.dumps(measure(ctx, L, prec, iters=a.iters, variant=v, batch=a.batch)),
                              flush=True)


if __name__ == "__main__":
    main()
