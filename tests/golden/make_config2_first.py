"""Writes config2_first.npz: the oracle's converged first increment of the
L = 256 shear workload (f = 0.20 Bernoulli voids, seed 0, first of 40
increments to 3x the void-free yield strain, matrix mu = 1, lambda = 1.5,
Y = 1, C0 = matrix, tolerances 1e-8, at most 60000 iterations): its record
(mean stress and strain, eta1, eta2, iterations, status) and the final local
strain at 4096 pixels drawn without replacement by numpy's default_rng(2).

Only the oracle is called.  Run from the repository root:
    python tests/golden/make_config2_first.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_0802_2488_gb300 import inputs  # noqa: E402

MAX_ITER = 60000
N_SAMPLE = 4096


def main():
    P = inputs.config2()
    mask = O.mask(P.L, P.f, P.seed)
    sol = O.solve(mask, O.material(), P.path[:1], tol_eq=1e-8, tol_macro=1e-8, max_iter=MAX_ITER, fields=True)
    idx = np.sort(np.random.default_rng(2).choice(P.L * P.L, N_SAMPLE, replace=False))
    r = sol.records[0]
    np.savez_compressed(os.path.join(HERE, "config2_first.npz"), pixels=idx,
                        eps=sol.eps.reshape(-1, 4)[idx], sig_mean=r["sig_mean"], eps_mean=r["eps_mean"],
                        eta1=r["eta1"], eta2=r["eta2"], iterations=r["iterations"], status=r["status"],
                        max_iter=MAX_ITER)
    print("iterations", int(r["iterations"]), "status", int(r["status"]), "eta1", float(r["eta1"]))


if __name__ == "__main__":
    main()
