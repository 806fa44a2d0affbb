"""Tiling variant 2 (the register-staged row and column passes, FP32
lattice sides 256 .. 4096, spectrum stored in the row transform's
digit-reversed order) against the oracle and against tiling 0.

Tolerances are those of the FP32 parity tests: one iteration chains four
FP32 transforms and the pixel update, so a few iterations stay within 2e-5
relative L2 of the FP64 oracle; the projection of Eqs. 2-3 within 3e-6."""
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
    c = B.Context(0)
    yield c
    c.close()


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_variant_2_exists_for_fp32_sides_256_to_4096_only():
    for L in (256, 512, 1024, 2048, 4096):
        assert B.epfft_supported_tiling(L, "fp32", 2)
        assert not B.epfft_supported_tiling(L, "fp64", 2)
    for L in (4, 16, 64, 128):
        assert not B.epfft_supported_tiling(L, "fp32", 2)
    assert B.epfft_supported_tiling(128, "fp32", 0) and B.epfft_supported_tiling(256, "fp64", 1)


@pytest.mark.parametrize("L,f,k", [(256, 0.2, 3), (512, 0.1, 2), (1024, 0.3, 2), (2048, 0.2, 1)])
def test_iterate_parity(ctx, L, f, k):
    B.epfft_set_tiling(ctx, L, "fp32", 2)
    try:
        mask = O.mask(L, f, 5)
        mat = O.material()
        E = np.array([0.45, 0.35, 0.0, 0.2])
        eps0 = inputs.random_strain(L, E, 0.3, seed=L + k)
        ref, lam = eps0.copy(), None
        for _ in range(k):
            ref, lam, _, _ = O.al_step(mask, mat, E, ref, lam)
        t = torch.tensor(eps0, dtype=torch.float32, device="cuda").contiguous()
        rec = B.epfft_iterate(ctx, B.Problem(L=L, precision="fp32", mask=mask), E, t, k)
        assert rec["iterations"] == k
        assert rel(t.cpu().numpy(), ref) < 2e-5, rel(t.cpu().numpy(), ref)
    finally:
        B.epfft_set_tiling(ctx, L, "fp32", 0)


@pytest.mark.parametrize("L", [256, 512, 4096])
def test_project_parity(ctx, L):
    B.epfft_set_tiling(ctx, L, "fp32", 2)
    try:
        rng = np.random.default_rng(L)
        p = rng.standard_normal((3, L, L))
        E = np.array([0.3, -0.2, 0.0, 0.15])
        pt = torch.tensor(p, dtype=torch.float32, device="cuda")
        e = B.epfft_project(ctx, L, "fp32", 1.5, 1.0, E, pt).cpu().numpy()
        if L <= 512:
            ph = np.stack([O.fft2(p[c], -1) for c in range(3)])
            eh = O.green_apply(L, 1.5, 1.0, E, ph)
            ref = np.stack([O.fft2(eh[c], +1).real / (L * L) for c in range(3)])
        else:  # the oracle's own DFT is slow here: tiling 0 is pinned against it at smaller sides
            B.epfft_set_tiling(ctx, L, "fp32", 0)
            ref = B.epfft_project(ctx, L, "fp32", 1.5, 1.0, E, pt).double().cpu().numpy()
        assert rel(e, ref) < 3e-6, rel(e, ref)
    finally:
        B.epfft_set_tiling(ctx, L, "fp32", 0)


@pytest.mark.parametrize("mode", ["cg1", "dg1"])
def test_general_operators(ctx, mode):
    """The column pass in its general form (continuum and symmetrized
    operators) on the digit-reversed column order."""
    L, k = 256, 2
    B.epfft_set_tiling(ctx, L, "fp32", 2)
    try:
        mask = O.mask(L, 0.2, 5)
        mat = O.material(green={"cg1": O.GREEN_CG1, "dg1": O.GREEN_DG1}[mode])
        E = np.array([0.45, 0.35, 0.0, 0.2])
        eps0 = inputs.random_strain(L, E, 0.3, seed=L + k)
        ref, lam = eps0.copy(), None
        for _ in range(k):
            ref, lam, _, _ = O.al_step(mask, mat, E, ref, lam)
        t = torch.tensor(eps0, dtype=torch.float32, device="cuda").contiguous()
        B.epfft_iterate(ctx, B.Problem(L=L, precision="fp32", mask=mask, green=mode), E, t, k)
        assert rel(t.cpu().numpy(), ref) < 2e-5
    finally:
        B.epfft_set_tiling(ctx, L, "fp32", 0)


def test_batched_solve_matches_tiling_0_and_is_independent_of_the_batch(ctx):
    """Four L = 256 lattices, three increments (iteration cap 40): the
    records of tiling 2 equal those of tiling 0 within the FP32 tolerance
    (same iteration counts, plastic counts within a few threshold pixels),
    and each solve of the batch gives the same bits alone."""
    L = 256
    path = inputs.load_path("shear", 3, 1.5)
    probs = [B.Problem(L=L, precision="fp32", void_fraction=f, seed=s, max_iter=40)
             for f, s in ((0.1, 0), (0.2, 1), (0.3, 2), (0.05, 3))]
    B.epfft_set_tiling(ctx, L, "fp32", 0)
    rc0, r0 = B.epfft_solve_batch(ctx, probs, [path] * 4)
    B.epfft_set_tiling(ctx, L, "fp32", 2)
    try:
        rc2, r2 = B.epfft_solve_batch(ctx, probs, [path] * 4)
        for a, b in zip(r0, r2):
            np.testing.assert_array_equal(a["iterations"], b["iterations"])
            assert rel(b["sig_mean"], a["sig_mean"]) < 1e-4
            assert np.abs(b["n_plastic"] - a["n_plastic"]).max() <= max(2, 0.01 * L * L)
        rc, alone = B.epfft_solve(ctx, probs[2], path)
        np.testing.assert_array_equal(alone["sig_mean"], r2[2]["sig_mean"])
        np.testing.assert_array_equal(alone["iterations"], r2[2]["iterations"])
    finally:
        B.epfft_set_tiling(ctx, L, "fp32", 0)


def test_displacement_matches_tiling_0(ctx):
    L = 512
    rng = np.random.default_rng(3)
    eps = torch.tensor(rng.standard_normal((L, L, 4)), dtype=torch.float32, device="cuda")
    B.epfft_set_tiling(ctx, L, "fp32", 0)
    u0 = B.epfft_displacement(ctx, L, "fp32", eps).double().cpu().numpy()
    B.epfft_set_tiling(ctx, L, "fp32", 2)
    try:
        u2 = B.epfft_displacement(ctx, L, "fp32", eps).double().cpu().numpy()
        assert rel(u2, u0) < 3e-6
    finally:
        B.epfft_set_tiling(ctx, L, "fp32", 0)


def test_autotune_times_all_three_tilings(ctx):
    chosen, ms = B.epfft_autotune(ctx, 512, "fp32", n_batch=16)
    # tilings 0-2 at L = 512; the on-chip schedule (3) is for sides up to 64
    assert len(ms) == 4 and all(m > 0 for m in ms[:3]) and ms[3] == 0 and ms[chosen] == min(ms[:3])
    chosen, ms = B.epfft_autotune(ctx, 256, "fp64")
    assert ms[2] == 0 and chosen in (0, 1)
    B.epfft_set_tiling(ctx, 512, "fp32", 0)
    B.epfft_set_tiling(ctx, 256, "fp64", 0)
