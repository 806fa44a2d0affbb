"""Mixed-precision solve: FP32 iterations to a switch tolerance, then FP64
iterations to the tolerance, per increment.  Its records are FP64 ones and
certify the tolerance the FP32 path alone cannot reach (its rounding
floor: eta1 of a few 1e-6 on a 256^2 lattice with voids); the fixed point
is that of the FP64 oracle.  Two solutions
that both meet eta2 < tol sit within tol / (1 - rho) of the fixed point, rho
the per-iteration contraction (here below 0.99, from the iteration counts),
so the macroscopic stresses agree within 100 tol = 1e-6 relative."""
import numpy as np
import pytest

import oracle as O
from paper_0802_2488_gb300 import binding as B
from paper_0802_2488_gb300 import inputs

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("tol_switch", [1e-6, 0.0])
@pytest.mark.parametrize("L,seed", [(16, 3), (32, 3)])
def test_refined_solve_certifies_the_tolerance(ctx, L, seed, tol_switch):
    """tol_switch = 0: the FP32 stage runs until it stalls at its floor."""
    path = inputs.load_path("shear", 3, 1.0)
    prob = B.Problem(L=L, precision="fp64", void_fraction=0.1, seed=seed, tol_eq=1e-8, tol_macro=1e-8,
                     max_iter=6000)
    rc, rec, rec32, f = B.epfft_solve_refined(ctx, prob, path, tol_switch=tol_switch, fields=True)
    assert rc == B.EPFFT_OK
    assert (rec["status"] == 0).all()
    assert (rec["eta1"] < 1e-8).all() and (rec["eta2"] < 1e-8).all()
    assert (rec32["iterations"] >= 1).all()
    ref = O.solve(O.mask(L, 0.1, seed), O.material(), path, tol_eq=1e-8, tol_macro=1e-8, max_iter=6000)
    assert ref.status == 0
    for k in range(len(path)):
        assert rel(rec["sig_mean"][k], ref.records["sig_mean"][k]) < 1e-6, k
    # the field outputs describe the final FP64 state
    mask = O.mask(L, 0.1, seed)
    _, pl = O.sigma(f.eps, mask, O.material())
    np.testing.assert_array_equal(f.plastic[-1], pl & (1 - mask))
    lab, n = O.label(f.plastic[-1])
    np.testing.assert_array_equal(f.labels[-1], lab)
    assert rec["n_clusters"][-1] == n


def test_refined_batch(ctx):
    """Three lattices advanced together (each leaves the FP32 stage on its
    own switch test): every one certified in FP64 and at the oracle's fixed
    point like a refined solve of its own."""
    L = 16
    path = inputs.load_path("shear", 2, 1.0)
    probs = [B.Problem(L=L, precision="fp64", void_fraction=0.1, seed=s, tol_eq=1e-8, tol_macro=1e-8, max_iter=6000)
             for s in (1, 2, 3)]
    rc, recs, recs32 = B.epfft_solve_refined_batch(ctx, probs, [path] * 3)
    assert rc == B.EPFFT_OK
    for s, r, r32 in zip((1, 2, 3), recs, recs32):
        assert (r["status"] == 0).all() and (r["eta1"] < 1e-8).all() and (r["eta2"] < 1e-8).all()
        assert (r32["iterations"] >= 1).all()
        ref = O.solve(O.mask(L, 0.1, s), O.material(), path, tol_eq=1e-8, tol_macro=1e-8, max_iter=6000)
        assert ref.status == 0
        assert rel(r["sig_mean"], ref.records["sig_mean"]) < 1e-6, s
    # unequal increment counts are refused
    with pytest.raises(B.EpfftError):
        B.epfft_solve_refined_batch(ctx, probs[:2], [path, path[:1]])


def test_refined_solve_arguments(ctx):
    path = inputs.load_path("shear", 1, 0.5)
    with pytest.raises(B.EpfftError):
        B.epfft_solve_refined(ctx, B.Problem(L=16, precision="fp32", void_fraction=0.1), path)
    with pytest.raises(B.EpfftError):
        B.epfft_solve_refined(ctx, B.Problem(L=16, void_fraction=0.1), path, tol_switch=-1.0)
