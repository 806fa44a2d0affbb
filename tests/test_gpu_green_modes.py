"""The other Green operators of Sec. 2 on the CUDA path against the oracle:
CG1 and DG1 iterations and solves, DG2 (four mirrored solves averaged) and
the CG2 average.  Tolerances as in test_gpu_parity: FP64 1e-12 per
iteration step and 1e-10 for converged solves, FP32 2e-5 for a few
iterations; integer results bit-exact."""
import numpy as np
import pytest

import oracle as O
from paper_0802_2488_gb300 import binding as B
from paper_0802_2488_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TDT = {"fp64": torch.float64, "fp32": torch.float32}
MODE = {"cg1": O.GREEN_CG1, "dg1": O.GREEN_DG1}


@pytest.fixture(scope="module")
def ctx():
    from paper_0802_2488_gb300 import build
    build.build()
    c = B.Context(0)
    yield c
    c.close()


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("mode", ["cg1", "dg1"])
@pytest.mark.parametrize("L,f,k", [(8, 0.2, 3), (32, 0.15, 4), (64, 0.1, 2), (256, 0.2, 2)])
def test_iterate_parity(ctx, mode, L, f, k, prec, tol):
    mask = O.mask(L, f, 5)
    mat = O.material(green=MODE[mode])
    E = np.array([0.45, 0.35, 0.0, 0.2])
    eps0 = inputs.random_strain(L, E, 0.3, seed=L + k)
    ref = eps0.copy()
    lam = None
    for _ in range(k):
        ref, lam, _, _ = O.al_step(mask, mat, E, ref, lam)
    t = torch.tensor(eps0, dtype=TDT[prec], device="cuda").contiguous()
    rec = B.epfft_iterate(ctx, B.Problem(L=L, precision=prec, mask=mask, green=mode), E, t, k)
    assert rec["iterations"] == k
    assert rel(t.cpu().numpy(), ref) < tol, rel(t.cpu().numpy(), ref)


@pytest.mark.parametrize("mode", ["cg1", "dg1"])
def test_solve_parity(ctx, mode):
    """Loading by increments; with CG1 and DG1 the equilibrium test is the
    fixed-point residual eta3, on both sides."""
    L = 16
    path = inputs.load_path("shear", 3, 1.5)
    mask = O.mask(L, 0.1, 3)
    ref = O.solve(mask, O.material(green=MODE[mode]), path, tol_eq=1e-8, tol_macro=1e-8, max_iter=4000, fields=True)
    prob = B.Problem(L=L, precision="fp64", void_fraction=0.1, seed=3, max_iter=4000, green=mode)
    rc, rec, f = B.epfft_solve(ctx, prob, path, fields=True)
    assert rc == (B.EPFFT_OK if ref.status == 0 else B.EPFFT_NOT_CONVERGED)
    np.testing.assert_array_equal(rec["iterations"], ref.records["iterations"])
    assert rel(rec["sig_mean"], ref.records["sig_mean"]) < 1e-10
    assert rel(f.eps, ref.eps) < 1e-10
    np.testing.assert_array_equal(f.plastic, ref.plastic)
    np.testing.assert_array_equal(f.labels, ref.labels)


@pytest.mark.parametrize("load", ["equibiaxial", "shear"])
def test_dg2_parity(ctx, load):
    L = 16
    path = inputs.load_path(load, 3, 1.5)
    mask = O.mask(L, 0.1, 4)
    kw = dict(tol_eq=1e-8, tol_macro=1e-8, max_iter=4000)
    ref = O.solve_dg2(mask, O.material(), path, **kw)
    prob = B.Problem(L=L, precision="fp64", mask=mask, max_iter=4000)
    rc, rec, f = B.epfft_solve_dg2(ctx, prob, path, fields=True)
    np.testing.assert_array_equal(rec["iterations"], ref.records["iterations"])
    assert rel(rec["sig_mean"], ref.records["sig_mean"]) < 1e-10
    assert rel(rec["eps_mean"], ref.records["eps_mean"]) < 1e-12
    assert rel(f.eps, ref.eps) < 1e-10
    # the plastic set of the averaged field (decided in FP64 on the device's
    # field by the oracle's law) and its clusters
    _, pl = O.sigma(f.eps, mask, O.material())
    np.testing.assert_array_equal(f.plastic, pl & (1 - mask))
    lab, n = O.label(f.plastic)
    np.testing.assert_array_equal(f.labels, lab)
    assert rec["n_clusters"][-1] == n and rec["n_plastic"][-1] == int(f.plastic.sum())
    assert (rec["n_clusters"][:-1] == -1).all()


def _symmetric_mask(L, f, seed):
    m = O.mask(L, f, seed)
    return np.maximum(m, O.mirror(m, (1,)))


def test_dg1_dg2_restore_mirror_symmetry(ctx):
    """Sec. 2: Eq. 3 gives asymmetric fields on a mirror-symmetric problem;
    DG1 and DG2 give symmetric ones."""
    L = 32
    mask = _symmetric_mask(L, 0.15, 5)
    path = inputs.load_path("equibiaxial", 2, 1.2)
    asym = lambda e: np.abs(e - O.mirror(e, (1,))).max() / np.abs(e).max()
    base = dict(L=L, precision="fp64", mask=mask, max_iter=3000, tol_eq=1e-9, tol_macro=1e-9)
    _, _, f3 = B.epfft_solve(ctx, B.Problem(**base), path, fields=True)
    _, _, f1 = B.epfft_solve(ctx, B.Problem(**base, green="dg1"), path, fields=True)
    _, _, f2 = B.epfft_solve_dg2(ctx, B.Problem(**base), path, fields=True)
    assert asym(f3.eps) > 1e-3
    assert asym(f1.eps) < 1e-11
    assert asym(f2.eps) < 1e-11


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-15), ("fp32", 1e-6)])
@pytest.mark.parametrize("L", [4, 64, 256])
def test_average5_parity(ctx, L, prec, tol):
    rng = np.random.default_rng(L)
    x = rng.standard_normal((L, L, 4))
    ref = O.avg5(x)
    t = torch.tensor(x, dtype=TDT[prec], device="cuda").contiguous()
    out = torch.empty_like(t)
    B.epfft_average5(ctx, L, prec, t, out)
    assert np.abs(out.cpu().numpy() - ref).max() < tol * (1 + np.abs(ref).max())


def test_mixed_operators_in_one_batch_match_solo(ctx):
    """A batch mixing Eq. 3 and CG1 / DG1 solves runs the general column pass;
    each solve's records equal those of the same solve alone (where an Eq. 3
    solve alone runs the specialised pass), bit for bit."""
    L = 16
    path = inputs.load_path("equibiaxial", 2, 1.2)
    probs = [B.Problem(L=L, precision=prec, void_fraction=0.1, seed=s, max_iter=600, green=g)
             for prec in ("fp64",) for s, g in ((1, "eq3"), (2, "cg1"), (3, "dg1"), (4, "eq3"))]
    _, recs = B.epfft_solve_batch(ctx, probs, [path] * len(probs))
    for p, r in zip(probs, recs):
        _, solo = B.epfft_solve(ctx, p, path)
        np.testing.assert_array_equal(r["iterations"], solo["iterations"])
        np.testing.assert_array_equal(r["sig_mean"], solo["sig_mean"])


@pytest.mark.parametrize("medium", ["one_void_cell", "bernoulli"])
@pytest.mark.parametrize("op", ["eq3", "dg2", "cg1", "dg1"])
def test_iteration_counts_under_one_criterion(ctx, op, medium):
    """The iteration-count comparison of Sec. 2 (every operator stopped on
    eta3 and eta2): the paper's matrix, equibiaxial loading past the yield
    strain, the one-void cell of Fig. 1 and a Bernoulli lattice; counts equal
    to the oracle's, macroscopic stress within 1e-10."""
    L = 32
    mask = inputs.one_void_cell(L, 0.1) if medium == "one_void_cell" else O.mask(L, 0.1, 0)
    path = inputs.load_path("equibiaxial", 3, 1.5, inputs.PAPER_MU, inputs.PAPER_YIELD)
    g = {"eq3": O.GREEN_EQ3, "dg2": O.GREEN_EQ3, "cg1": O.GREEN_CG1, "dg1": O.GREEN_DG1}[op]
    mat = O.material(lam=inputs.PAPER_LAMBDA, mu=inputs.PAPER_MU, Y=inputs.PAPER_YIELD, green=g)
    kw = dict(tol_eq=1e-5, tol_macro=1e-5, max_iter=20000, eq_test=O.EQ_FIXED_POINT)
    ref = (O.solve_dg2 if op == "dg2" else O.solve)(mask, mat, path, **kw).records
    prob = B.Problem(L=L, precision="fp64", mask=mask, mu=inputs.PAPER_MU, lambda_=inputs.PAPER_LAMBDA,
                     yield_stress=inputs.PAPER_YIELD, tol_eq=1e-5, tol_macro=1e-5, max_iter=20000,
                     green="eq3" if op == "dg2" else op, eq_test="fixed_point")
    rc, rec = (B.epfft_solve_dg2 if op == "dg2" else B.epfft_solve)(ctx, prob, path)
    assert rc == B.EPFFT_OK and (ref["status"] == 0).all()
    np.testing.assert_array_equal(rec["iterations"], ref["iterations"])
    assert rel(rec["sig_mean"], ref["sig_mean"]) < 1e-10
