"""Converged FP64 solve at the shear workload's lattice size (L = 256,
f = 0.20, seed 0; first of its 40 increments, tolerances 1e-8) against the
oracle's converged solve stored in tests/golden/config2_first.npz (written by
tests/golden/make_config2_first.py, which calls only the oracle): the same
number of iterations (within two, where the stopping test crosses its
threshold at rounding level), the macroscopic stress within 1e-10 relative,
and the final local strain at the stored 4096 sampled pixels within 1e-10
relative L2 (1e-8 if the iteration counts differ)."""
import os

import numpy as np
import pytest

from paper_0802_2488_gb300 import binding as B
from paper_0802_2488_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_first_increment_of_the_shear_workload_converges_like_the_oracle():
    from paper_0802_2488_gb300 import build
    build.build()
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "config2_first.npz"))
    P = inputs.config2()
    prob = B.Problem(L=P.L, precision="fp64", void_fraction=P.f, seed=P.seed, tol_eq=1e-8, tol_macro=1e-8,
                     max_iter=int(g["max_iter"]))
    with B.Context(0) as ctx:
        rc, rec, f = B.epfft_solve(ctx, prob, P.path[:1], fields=True)
    assert int(g["status"]) == 0 and rc == B.EPFFT_OK and rec["status"][0] == 0
    d_it = abs(int(rec["iterations"][0]) - int(g["iterations"]))
    assert d_it <= 2, (int(rec["iterations"][0]), int(g["iterations"]))
    s_err = np.linalg.norm(rec["sig_mean"][0] - g["sig_mean"]) / np.linalg.norm(g["sig_mean"])
    eps = f.eps.reshape(-1, 4)[g["pixels"]]
    e_err = np.linalg.norm(eps - g["eps"]) / np.linalg.norm(g["eps"])
    bound = 1e-10 if d_it == 0 else 1e-8
    assert s_err < bound and e_err < bound, (d_it, s_err, e_err)
    assert rec["eta1"][0] < 1e-8 and rec["eta2"][0] < 1e-8
