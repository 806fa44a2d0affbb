"""The on-chip schedule (tiling 3: FP32, L = 16 .. 64, one CTA runs a whole
solve with the spectrum in shared memory) against the two-pass loop and the
oracle.

Its transforms, Green operator of Eq. 3 and pixel update evaluate the same
formulas per element as the two passes of tiling 0 (the same plans and
tables); the compiler's fused multiply-add choices and the order of the CTA
sums differ.  So a fixed number of iterations (tolerances 0, every increment
at its cap) gives the two-pass loop's strain to FP32 rounding; solves to a
tolerance the FP32 form reaches agree with the oracle within FP32 error; a
batch gives each solve's result bit for bit as the solve alone.
"""
import numpy as np
import pytest

import oracle as O
from paper_0802_2488_gb300 import binding as B
from paper_0802_2488_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_0802_2488_gb300 import build
    build.build()
    with B.Context(0) as c:
        yield c


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def solve_with(ctx, tiling, prob, path, fields=True):
    B.epfft_set_tiling(ctx, prob.L, "fp32", tiling)
    try:
        return B.epfft_solve(ctx, prob, path, fields=fields)
    finally:
        B.epfft_set_tiling(ctx, prob.L, "fp32", 0)


@pytest.mark.parametrize("L", [16, 32, 64])
@pytest.mark.parametrize("load", ["equibiaxial", "shear"])
def test_fixed_iterations_agree_with_the_two_pass_loop(ctx, L, load):
    path = inputs.load_path(load, 3, 2.0)
    prob = B.Problem(L=L, precision="fp32", void_fraction=0.15, seed=L, tol_eq=0.0, tol_macro=0.0, max_iter=40)
    rc0, r0, f0 = solve_with(ctx, 0, prob, path)
    rc3, r3, f3 = solve_with(ctx, 3, prob, path)
    assert B.epfft_last_stats(ctx)["kernel_launches"] <= 1 + 1 + 4  # mask, the solve, labelling
    np.testing.assert_array_equal(r3["iterations"], r0["iterations"])
    assert rel(f3.eps, f0.eps) < 1e-5, rel(f3.eps, f0.eps)
    # plastic flags may differ where a pixel sits at the threshold to rounding
    assert (f3.plastic != f0.plastic).sum() <= max(2, f0.plastic.size // 1000)
    for k in range(len(path)):
        np.testing.assert_array_equal(f3.labels[k], O.label(f3.plastic[k])[0])
    assert rel(r3["sig_mean"], r0["sig_mean"]) < 1e-5
    assert rel(r3["eta1"], r0["eta1"]) < 1e-3


@pytest.mark.parametrize("L", [16, 32, 64])
def test_solve_to_tolerance_matches_the_oracle(ctx, L):
    # shear to 1.5x yield in 3 increments: the oracle converges to 1e-5 within
    # 9000 iterations per increment at these sides
    path = inputs.load_path("shear", 3, 1.5)
    mask = O.mask(L, 0.1, 3)
    ref = O.solve(mask, O.material(), path, tol_eq=1e-5, tol_macro=1e-5, max_iter=20000, fields=True)
    assert ref.status == 0
    prob = B.Problem(L=L, precision="fp32", mask=mask, tol_eq=1e-5, tol_macro=1e-5, max_iter=20000)
    rc, rec, f = solve_with(ctx, 3, prob, path)
    assert rc == B.EPFFT_OK
    assert (np.abs(rec["iterations"] - ref.records["iterations"]) <= 0.02 * ref.records["iterations"] + 2).all()
    assert rel(rec["sig_mean"], ref.records["sig_mean"]) < 1e-4
    assert rel(f.eps, ref.eps) < 1e-3
    for k in range(len(path)):
        np.testing.assert_array_equal(f.labels[k], O.label(f.plastic[k])[0])


def test_batch_equals_the_solves_alone(ctx):
    path = inputs.load_path("shear", 3, 1.5)
    probs = [B.Problem(L=32, precision="fp32", void_fraction=0.1, seed=s, tol_eq=1e-5, tol_macro=1e-5, max_iter=5000)
             for s in (1, 2, 3, 4)]
    B.epfft_set_tiling(ctx, 32, "fp32", 3)
    try:
        alone = [B.epfft_solve(ctx, p, path, fields=True) for p in probs]
        rc, recs, fs = B.epfft_solve_batch(ctx, probs, [path] * 4, fields=True)
    finally:
        B.epfft_set_tiling(ctx, 32, "fp32", 0)
    for (r0, rec0, f0), rec, f in zip(alone, recs, fs):
        np.testing.assert_array_equal(rec0, rec)
        np.testing.assert_array_equal(f0.eps, f.eps)


def test_mixed_call_with_on_chip_and_two_pass_groups(ctx):
    """One epfft_solve_batch call whose L = 32 FP32 group runs on the
    on-chip schedule (on a stream of its own, while the graph of the other
    groups runs) and whose L = 128 FP32 and L = 64 FP64 groups run the two
    passes: every result equals the same problem solved alone."""
    path = inputs.load_path("shear", 3, 1.5)
    probs = [B.Problem(L=32, precision="fp32", void_fraction=0.1, seed=s, tol_eq=1e-5, tol_macro=1e-5, max_iter=5000)
             for s in (5, 6)]
    probs += [B.Problem(L=128, precision="fp32", void_fraction=0.2, seed=7, max_iter=60),
              B.Problem(L=64, precision="fp64", void_fraction=0.15, seed=8, max_iter=80)]
    B.epfft_set_tiling(ctx, 32, "fp32", 3)
    try:
        alone = [B.epfft_solve(ctx, p, path, fields=True) for p in probs]
        rc, recs, fs = B.epfft_solve_batch(ctx, probs, [path] * len(probs), fields=True)
    finally:
        B.epfft_set_tiling(ctx, 32, "fp32", 0)
    for (r0, rec0, f0), rec, f in zip(alone, recs, fs):
        np.testing.assert_array_equal(rec0, rec)
        np.testing.assert_array_equal(f0.eps, f.eps)


def test_autotune_times_the_on_chip_schedule(ctx):
    chosen, ms = B.epfft_autotune(ctx, 64, "fp32", n_batch=152)
    assert ms[3] > 0.0 and ms[2] == 0.0
    assert chosen in (0, 1, 3)
    B.epfft_set_tiling(ctx, 64, "fp32", 0)
