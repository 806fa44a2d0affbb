"""The displacement field of Sec. 2 on the CUDA path against the oracle and
against a known displacement: a periodic displacement differenced with the
forward differences of Eq. 1 comes back (minus its mean), through the
frequencies where k1^2 + k2^2 vanishes too; an arbitrary (incompatible)
strain gives the oracle's field.  FP64 to round-off, FP32 within 1e-5 of
the field's scale."""
import numpy as np
import pytest

import oracle as O
from paper_0802_2488_gb300 import binding as B
from paper_0802_2488_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TDT = {"fp64": torch.float64, "fp32": torch.float32}
TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def ctx():
    from paper_0802_2488_gb300 import build
    build.build()
    c = B.Context(0)
    yield c
    c.close()


def strain_of(u):
    d1 = lambda f: np.roll(f, -1, axis=1) - f
    d2 = lambda f: np.roll(f, -1, axis=0) - f
    e = np.zeros(u.shape[:2] + (4,))
    e[..., 0] = d1(u[..., 0])
    e[..., 1] = d2(u[..., 1])
    e[..., 3] = 0.5 * (d2(u[..., 0]) + d1(u[..., 1]))
    return e


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("L", [4, 16, 64, 256, 1024])
def test_known_displacement_comes_back(ctx, L, prec):
    rng = np.random.default_rng(L + 1)
    u = rng.standard_normal((L, L, 2))
    e = torch.tensor(strain_of(u), dtype=TDT[prec], device="cuda").contiguous()
    got = B.epfft_displacement(ctx, L, prec, e).cpu().numpy()
    ref = u - u.mean(axis=(0, 1))
    assert np.abs(got - ref).max() < TOL[prec] * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("L", [8, 128])
def test_incompatible_strain_matches_oracle(ctx, L, prec):
    rng = np.random.default_rng(L)
    e = rng.standard_normal((L, L, 4))
    ref = O.displacement(e)
    got = B.epfft_displacement(ctx, L, prec, torch.tensor(e, dtype=TDT[prec], device="cuda")).cpu().numpy()
    assert np.abs(got - ref).max() < TOL[prec] * np.abs(ref).max()


def test_converged_solve_field(ctx):
    """The final strain of a converged solve (L = 32, f = 0.1, seed 3, the
    three-increment shear path, tolerance 1e-8) is compatible up to the
    stopping tolerance: the displacement reproduces its forward-difference
    strain less the mean (the oracle's own field does to 2.5e-10 relative)."""
    L = 32
    path = inputs.load_path("shear", 3, 1.0)
    rc, rec, f = B.epfft_solve(ctx, B.Problem(L=L, precision="fp64", void_fraction=0.1, seed=3, tol_eq=1e-8,
                                              tol_macro=1e-8, max_iter=4000), path, fields=True)
    assert rc == B.EPFFT_OK
    u = B.epfft_displacement(ctx, L, "fp64", torch.tensor(f.eps, device="cuda")).cpu().numpy()
    back = strain_of(u)
    fluct = f.eps.copy()
    fluct[..., (0, 1, 3)] -= fluct[..., (0, 1, 3)].mean(axis=(0, 1))
    assert np.abs(back[..., (0, 1, 3)] - fluct[..., (0, 1, 3)]).max() < 1e-8 * np.abs(f.eps).max()
