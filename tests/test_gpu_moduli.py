"""Effective moduli (elastic matrix, Eqs. 5-6) and the equivalent strain of
Fig. 1 on the CUDA path against the oracle; the Eqs. 5-6 curve of a solve."""
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


@pytest.mark.parametrize("L,f", [(16, 0.0), (32, 0.1), (64, 0.3)])
def test_effective_moduli_parity(ctx, L, f):
    mask = O.mask(L, f, 2)
    K, mu = B.epfft_effective_moduli(ctx, B.Problem(L=L, precision="fp64", mask=mask, tol_eq=1e-10,
                                                    tol_macro=1e-10, max_iter=20000))
    rK, rmu = O.effective_moduli(mask, O.material(), tol=1e-10, max_iter=20000)
    assert abs(K - rK) < 1e-9 * rK and abs(mu - rmu) < 1e-9 * rmu
    if f == 0.0:
        assert abs(K - 5.0) < 1e-12 and abs(mu - 1.0) < 1e-12


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-15), ("fp32", 1e-6)])
def test_eps_eq_parity(ctx, prec, tol):
    L = 64
    rng = np.random.default_rng(1)
    e = rng.standard_normal((L, L, 4))
    t = torch.tensor(e, dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda").contiguous()
    got = B.epfft_eps_eq(ctx, L, prec, t).cpu().numpy()
    ref = O.eps_eq(e)
    assert np.abs(got - ref).max() < tol * (1 + ref.max())


def test_empirical_curve_of_a_solve(ctx):
    """Eq. 6 on a shear solve: indicators from the device clusters, mu~ from
    the device, the fit from the library; the same numbers as the oracle's
    chain on the device's flags and records."""
    L = 32
    path = inputs.load_path("shear", 8, 3.0)
    prob = B.Problem(L=L, precision="fp64", void_fraction=0.1, seed=2, max_iter=300)
    rc, rec, f = B.epfft_solve(ctx, prob, path, fields=True)
    mask = O.mask(L, 0.1, 2)
    st = B.epfft_void_plastic(ctx, mask, f.plastic)
    ind = B.epfft_indicators(rec, st, L, "shear")
    K, mu = B.epfft_effective_moduli(ctx, B.Problem(L=L, precision="fp64", void_fraction=0.1, seed=2,
                                                    tol_eq=1e-10, tol_macro=1e-10, max_iter=20000))
    a, fit = B.epfft_empirical_curve(ind, st, L, mu, "shear")
    ra, rfit = O.empirical_curve(O.indicators(rec, st, L, "shear"), st, L, mu, "shear")
    assert abs(a - ra) < 1e-10 * max(1, abs(ra))
    np.testing.assert_allclose(fit, rfit, rtol=1e-10, atol=1e-12)
    assert np.isfinite(fit).all()
