"""Writes config1_oracle.json: the oracle's per-increment records for the
L = 64 equibiaxial workload (f = 0.10 Bernoulli voids, seed 0, 20 increments
to 2x the void-free yield strain, matrix mu = 1, lambda = 1.5, Y = 1, C0 =
matrix, tolerances 1e-8, at most 20000 iterations per increment), and
config1_fields.npz: the final local strain of the whole path and, for each
increment k that converges (status 0), the final strain of the solve of the
path's first k increments (the same arithmetic, so the state the full solve
holds after increment k).

Only the oracle is called.  Run from the repository root:
    python tests/golden/make_config1.py [--fields-only]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_0802_2488_gb300 import inputs  # noqa: E402

MAX_ITER = 20000


def main():
    P = inputs.config1()
    mask = O.mask(P.L, P.f, P.seed)
    t = time.time()
    sol = O.solve(mask, O.material(), P.path, tol_eq=1e-8, tol_macro=1e-8, max_iter=MAX_ITER, fields=True)
    rec = sol.records
    out = {
        "source": "oracle/oracle.c orc_solve, written by tests/golden/make_config1.py",
        "problem": {"L": P.L, "f": P.f, "seed": P.seed, "mode": P.mode, "n_inc": P.n_inc,
                    "multiple": P.multiple, "tol_eq": 1e-8, "tol_macro": 1e-8, "max_iter": MAX_ITER},
        "oracle_seconds": time.time() - t,
        "records": [{"sig_mean": r["sig_mean"].tolist(), "eps_mean": r["eps_mean"].tolist(),
                     "eta1": float(r["eta1"]), "eta2": float(r["eta2"]), "eta3": float(r["eta3"]),
                     "iterations": int(r["iterations"]), "n_plastic": int(r["n_plastic"]),
                     "n_clusters": int(r["n_clusters"]), "status": int(r["status"])} for r in rec],
        "void_pixels": int(mask.sum()),
    }
    with open(os.path.join(HERE, "config1_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    write_fields(P, mask, sol)


def write_fields(P, mask, sol=None):
    if sol is None:
        sol = O.solve(mask, O.material(), P.path, tol_eq=1e-8, tol_macro=1e-8, max_iter=MAX_ITER, fields=True)
    fields = {"final": sol.eps}
    for k in range(P.n_inc):
        if sol.records["status"][k] != 0:
            continue
        pre = O.solve(mask, O.material(), P.path[:k + 1], tol_eq=1e-8, tol_macro=1e-8, max_iter=MAX_ITER,
                      fields=True)
        assert (pre.records["iterations"] == sol.records["iterations"][:k + 1]).all()
        fields[f"after_{k + 1}"] = pre.eps
    np.savez_compressed(os.path.join(HERE, "config1_fields.npz"), **fields)


if __name__ == "__main__":
    if "--fields-only" in sys.argv:
        P = inputs.config1()
        write_fields(P, O.mask(P.L, P.f, P.seed))
    else:
        main()
