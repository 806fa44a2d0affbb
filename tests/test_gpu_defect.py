"""The defect-correction form ('fp32_defect', EPFFT_FP32_DEFECT) against the
oracle.

The form iterates in FP32 on the differences of strain and stress from an
FP64 reference state, which a refresh (FP64 transforms, every
`epfft_set_defect_refresh` loop steps and after each warm start) moves to the
current iterate.  Three properties pin it:

* its FP32 rounding scales with the iterate's distance from the last
  refresh: near the fixed point, with a refresh before every iteration, the
  iterates are the oracle's FP64 ones within 1e-11 (the plain FP32 form is
  off by its FP32 state); from a generic state, and without refreshes, they
  stay within the FP32 form's 2e-5;
* with the default refresh it converges where the FP32 form cannot: the
  shear workload's first increment (L = 256, f = 0.2) reaches eta1, eta2 <
  1e-8, and the oracle, evaluating Eq. 1's divergence of the returned strain
  field itself, confirms eta1 < 1e-8; the macroscopic stress agrees with the
  oracle's converged solve (tests/golden/config2_first.npz) within 1e-6.

A batch and a call mixing precisions give each solve's result bit for bit
as the solve alone.
"""
import os

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


def oracle_iterate(mask, mat, E, eps, k):
    lam = None
    for _ in range(k):
        eps, lam, e, _ = O.al_step(mask, mat, E, eps, lam)
    return eps


def eta1_of(mask, eps):
    """eta1 of Sec. 2 (Eq. 1's backward divergence of sigma(eps)) evaluated
    by the oracle on a returned strain field."""
    st = O.stats(mask, O.material(), eps)
    s = st.sig_mean
    return float(np.sqrt(st.div2_mean / (s[0] ** 2 + s[1] ** 2 + 2 * s[3] ** 2)))


def test_supported_sides_and_tilings():
    assert B.epfft_supported(256, "fp32_defect") and B.epfft_supported(4096, "fp32_defect")
    assert not B.epfft_supported(8192, "fp32_defect")
    assert B.epfft_supported_tiling(256, "fp32_defect", 0) and B.epfft_supported_tiling(256, "fp32_defect", 1)
    assert not B.epfft_supported_tiling(512, "fp32_defect", 2)


@pytest.mark.parametrize("green", ["eq3", "cg1"])
def test_near_the_fixed_point_the_iterates_are_the_fp64_ones(ctx, green):
    """The FP32 rounding of the defect form scales with how far the iterate
    moved since the last refresh.  From the oracle's solution (tolerances
    1e-11) perturbed by 1e-6, with a refresh before every iteration, five
    iterations agree with the oracle's FP64 iterations within 1e-11, where the
    plain FP32 form, whose state is rounded to FP32, is off by about 1e-8."""
    L, f, k = 32, 0.15, 5
    mask = O.mask(L, f, 5)
    mat = O.material(green=O.GREEN_EQ3 if green == "eq3" else O.GREEN_CG1)
    E = np.array([0.45, 0.35, 0.0, 0.2])
    sol = O.solve(mask, mat, E[None], tol_eq=1e-11, tol_macro=1e-11, max_iter=200000, fields=True)
    assert sol.status == 0
    eps0 = sol.eps + inputs.random_strain(L, np.zeros(4), 1e-6, seed=3)
    ref = oracle_iterate(mask, mat, E, eps0.copy(), k)
    prob = B.Problem(L=L, precision="fp32_defect", mask=mask, green=green)
    B.epfft_set_defect_refresh(ctx, 1)
    try:
        t = torch.tensor(eps0, dtype=torch.float64, device="cuda").contiguous()
        rec = B.epfft_iterate(ctx, prob, E, t, k)
    finally:
        B.epfft_set_defect_refresh(ctx, 256)
    assert rec["iterations"] == k
    err = rel(t.cpu().numpy(), ref)
    assert err < 1e-11, err
    t32 = torch.tensor(eps0, dtype=torch.float32, device="cuda").contiguous()
    B.epfft_iterate(ctx, B.Problem(L=L, precision="fp32", mask=mask, green=green), E, t32, k)
    assert rel(t32.cpu().numpy().astype(np.float64), ref) > 1e-9


@pytest.mark.parametrize("L,f,k", [(8, 0.2, 3), (64, 0.10, 4), (256, 0.2, 3), (512, 0.1, 2)])
def test_refresh_every_step_from_a_generic_state(ctx, L, f, k):
    """From a generic state (noise 0.3) the iteration's steps are large and
    the FP32 differences carry FP32 rounding: within the FP32 form's 2e-5."""
    mask = O.mask(L, f, 5)
    mat = O.material()
    E = np.array([0.45, 0.35, 0.0, 0.2])
    eps0 = inputs.random_strain(L, E, 0.3, seed=L + k)
    ref = oracle_iterate(mask, mat, E, eps0.copy(), k)
    B.epfft_set_defect_refresh(ctx, 1)
    try:
        t = torch.tensor(eps0, dtype=torch.float64, device="cuda").contiguous()
        rec = B.epfft_iterate(ctx, B.Problem(L=L, precision="fp32_defect", mask=mask), E, t, k)
    finally:
        B.epfft_set_defect_refresh(ctx, 256)
    assert rec["iterations"] == k
    assert rel(t.cpu().numpy(), ref) < 2e-5, rel(t.cpu().numpy(), ref)


@pytest.mark.parametrize("L,f,k", [(8, 0.2, 3), (64, 0.10, 4), (128, 0.3, 2), (512, 0.2, 2)])
def test_without_refresh_it_is_the_fp32_transform(ctx, L, f, k):
    mask = O.mask(L, f, 5)
    mat = O.material()
    E = np.array([0.45, 0.35, 0.0, 0.2])
    eps0 = inputs.random_strain(L, E, 0.3, seed=L + k)
    ref = oracle_iterate(mask, mat, E, eps0.copy(), k)
    B.epfft_set_defect_refresh(ctx, 1 << 20)
    try:
        t = torch.tensor(eps0, dtype=torch.float64, device="cuda").contiguous()
        B.epfft_iterate(ctx, B.Problem(L=L, precision="fp32_defect", mask=mask), E, t, k)
    finally:
        B.epfft_set_defect_refresh(ctx, 256)
    err = rel(t.cpu().numpy(), ref)
    assert err < 2e-5, err
    assert err > 1e-12  # the FP32 transforms did run


def test_shear_workload_first_increment_certified_at_1e8(ctx):
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "config2_first.npz"))
    P = inputs.config2()
    prob = B.Problem(L=P.L, precision="fp32_defect", void_fraction=P.f, seed=P.seed, tol_eq=1e-8,
                     tol_macro=1e-8, max_iter=int(g["max_iter"]))
    rc, rec, f = B.epfft_solve(ctx, prob, P.path[:1], fields=True)
    assert rc == B.EPFFT_OK and rec["status"][0] == 0
    assert rec["eta1"][0] < 1e-8 and rec["eta2"][0] < 1e-8
    assert f.eps.dtype == np.float64
    mask = O.mask(P.L, P.f, P.seed)
    e1 = eta1_of(mask, f.eps)
    assert e1 < 1e-8, e1
    assert abs(e1 - rec["eta1"][0]) < 1e-3 * rec["eta1"][0]
    assert rel(rec["sig_mean"][0], g["sig_mean"]) < 1e-6
    # the plastic flags and clusters are those of the returned field
    pl = O.stats(mask, O.material(), f.eps).plastic
    np.testing.assert_array_equal(f.plastic[0], pl)
    np.testing.assert_array_equal(f.labels[0], O.label(pl)[0])


def test_small_solve_by_increments_against_the_oracle(ctx):
    L = 16
    path = inputs.load_path("equibiaxial", 4, 1.5)
    mask = O.mask(L, 0.1, 3)
    # the oracle needs 1038, 5551, 13218 and 20495 iterations
    ref = O.solve(mask, O.material(), path, tol_eq=1e-8, tol_macro=1e-8, max_iter=40000, fields=True)
    prob = B.Problem(L=L, precision="fp32_defect", void_fraction=0.1, seed=3, max_iter=40000)
    rc, rec, f = B.epfft_solve(ctx, prob, path, fields=True)
    assert ref.status == 0 and rc == B.EPFFT_OK
    assert (rec["eta1"] < 1e-8).all() and (rec["eta2"] < 1e-8).all()
    assert rel(rec["sig_mean"], ref.records["sig_mean"]) < 1e-6
    assert rel(f.eps, ref.eps) < 1e-5
    assert eta1_of(mask, f.eps) < 1e-8


def test_batch_and_mixed_call_equal_the_solves_alone(ctx):
    path = inputs.load_path("shear", 3, 1.5)
    probs = [B.Problem(L=32, precision="fp32_defect", void_fraction=0.15, seed=s, max_iter=3000) for s in (1, 2, 3)]
    alone = [B.epfft_solve(ctx, p, path, fields=True) for p in probs]
    rc, recs, fs = B.epfft_solve_batch(ctx, probs, [path] * 3, fields=True)
    for (r0, rec0, f0), rec, f in zip(alone, recs, fs):
        np.testing.assert_array_equal(rec0, rec)
        np.testing.assert_array_equal(f0.eps, f.eps)
    others = [B.Problem(L=64, precision="fp64", void_fraction=0.1, seed=4, max_iter=3000),
              B.Problem(L=16, precision="fp32", void_fraction=0.1, seed=5, max_iter=3000)]
    solo_o = [B.epfft_solve(ctx, p, path) for p in others]
    rc, recs, fs = B.epfft_solve_batch(ctx, probs[:1] + others, [path] * 3, fields=True)
    np.testing.assert_array_equal(alone[0][1], recs[0])
    np.testing.assert_array_equal(alone[0][2].eps, fs[0].eps)
    for (r0, rec0), rec in zip(solo_o, recs[1:]):
        np.testing.assert_array_equal(rec0, rec)


def test_served_defect_solve_is_certified(ctx):
    L = 32
    path = inputs.load_path("equibiaxial", 3, 1.5)
    # the oracle needs 2934, 10859 and 20975 iterations
    prob = B.Problem(L=L, precision="fp32_defect", void_fraction=0.1, seed=9, max_iter=60000)
    B.epfft_serve_open(ctx, 1 << 30, 4, 64)
    try:
        t = B.epfft_submit(ctx, prob, path, want_eps=True)
        r = None
        for _ in range(10000):
            B.epfft_serve_step(ctx)
            r = B.epfft_poll(ctx, t, prob, len(path), want_eps=True)
            if r is not None:
                break
    finally:
        B.epfft_serve_close(ctx)
    assert r is not None
    rc, rec, eps, _ = r
    assert rc == B.EPFFT_OK and (rec["status"] == 0).all()
    assert (rec["eta1"] < 1e-8).all() and eps.dtype == np.float64
    assert eta1_of(O.mask(L, 0.1, 9), eps) < 1e-8


@pytest.mark.parametrize("load", ["equibiaxial", "shear"])
def test_dg2_in_the_defect_form(ctx, load):
    """DG2 (Sec. 2: four solves with the mirrored operators, fields
    averaged) with every member in the defect form, against the oracle's
    FP64 DG2 at the same tolerances (all increments converge within the
    cap): the macroscopic stress within 1e-6, the averaged field within
    1e-5, the iteration counts within 1 %, and the plastic set and clusters
    of the averaged field those of the oracle's law on it."""
    L = 16
    path = inputs.load_path(load, 3, 1.5)
    mask = O.mask(L, 0.1, 4)
    ref = O.solve_dg2(mask, O.material(), path, tol_eq=1e-8, tol_macro=1e-8, max_iter=30000)
    assert (ref.records["status"] == 0).all()
    prob = B.Problem(L=L, precision="fp32_defect", mask=mask, max_iter=30000)
    rc, rec, f = B.epfft_solve_dg2(ctx, prob, path, fields=True)
    assert rc == B.EPFFT_OK and (rec["status"] == 0).all()
    assert (np.abs(rec["iterations"] - ref.records["iterations"]) <= 0.01 * ref.records["iterations"]).all()
    assert rel(rec["sig_mean"], ref.records["sig_mean"]) < 1e-6
    assert rel(f.eps, ref.eps) < 1e-5
    _, pl = O.sigma(f.eps, mask, O.material())
    np.testing.assert_array_equal(f.plastic, pl & (1 - mask))
    lab, n = O.label(f.plastic)
    np.testing.assert_array_equal(f.labels, lab)
