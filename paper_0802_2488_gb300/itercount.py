"""Iteration counts of the Green operators of Sec. 2 on the paper's two media,
all stopped by one criterion (the fixed-point residual eta3 and the
macroscopic change eta2, both below `tol`), so that the counts compare the
operators and not their tests.  Sec. 2 states that DG2 needs fewer iterations
than CG1 on a periodic void lattice and on the pixelwise disordered medium
(tolerances about 1e-5, L = 512 to 2048).

    python -m paper_0802_2488_gb300.itercount --L 512 --precision fp32 --tol 1e-5

Media: the periodic cell of Fig. 1 (one circular void, f = 0.1) and the
Bernoulli lattice (f = 0.1, seed 0), with the paper's matrix (K = 1,
mu = 0.4, Y = 0.5) under equibiaxial loading ramped to `--multiple` times
the void-free yield strain.  Operators: Eq. 3 alone, DG2 (its four members,
reported per member), CG1 and DG1.  One JSON line per medium and operator.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import binding as B
from . import inputs


def media(L: int):
    return {"one_void_cell": inputs.one_void_cell(L, 0.1), "bernoulli": None}


def run(ctx, L: int, precision: str, tol: float, n_inc: int, multiple: float, max_iter: int,
        operators=("eq3", "dg2", "cg1", "dg1")):
    path = inputs.load_path("equibiaxial", n_inc, multiple, inputs.PAPER_MU, inputs.PAPER_YIELD)
    out = []
    for name, mask in media(L).items():
        for op in operators:
            prob = B.Problem(L=L, precision=precision, void_fraction=0.1, seed=0, mask=mask,
                             mu=inputs.PAPER_MU, lambda_=inputs.PAPER_LAMBDA, yield_stress=inputs.PAPER_YIELD,
                             tol_eq=tol, tol_macro=tol, max_iter=max_iter,
                             green="eq3" if op == "dg2" else op, eq_test="fixed_point")
            t0 = time.perf_counter()
            if op == "dg2":
                rc, rec = B.epfft_solve_dg2(ctx, prob, path)
                members = 4
            else:
                rc, rec = B.epfft_solve(ctx, prob, path)
                members = 1
            dt = time.perf_counter() - t0
            its = rec["iterations"].astype(np.int64)
            out.append({
                "medium": name, "operator": op, "L": L, "precision": precision, "tol": tol,
                "n_inc": n_inc, "multiple": multiple,
                "iterations_per_increment": (its / members).tolist(),
                "iterations_per_solve": float(its.sum() / members),
                "members": members,
                "converged": bool((rec["status"] == 0).all()),
                "sig11_final": float(rec["sig_mean"][-1][0]),
                "seconds": dt,
            })
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--L", type=int, default=512)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-5)
    ap.add_argument("--n-inc", type=int, default=5)
    ap.add_argument("--multiple", type=float, default=1.5)
    ap.add_argument("--max-iter", type=int, default=20000)
    ap.add_argument("--operators", nargs="+", default=["eq3", "dg2", "cg1", "dg1"])
    a = ap.parse_args(argv)
    ctx = B.Context(0)
    try:
        for r in run(ctx, a.L, a.precision, a.tol, a.n_inc, a.multiple, a.max_iter, a.operators):
            print(json.dumps(r), flush=True)
    finally:
        ctx.close()


if __name__ == "__main__":
    main()
