"""Pins of the oracle's effective moduli, the empirical formulas of Eqs. 5-6
and the equivalent strain of Fig. 1: closed forms of the void-free matrix,
the Voigt bound, recovery of a planted fitting number, and closed-form
equivalent strains."""
import numpy as np
import pytest

import oracle as O


def test_effective_moduli_void_free_closed_form():
    K, mu = O.effective_moduli(np.zeros((8, 8), np.uint8), O.material(lam=1.5, mu=1.0))
    assert abs(K - 5.0) < 1e-12 and abs(mu - 1.0) < 1e-12
    K, mu = O.effective_moduli(np.zeros((8, 8), np.uint8), O.material(lam=11 / 15, mu=0.4))
    assert abs(K - 2 * (11 / 15 + 0.4)) < 1e-12 and abs(mu - 0.4) < 1e-12


@pytest.mark.parametrize("f", [0.05, 0.2])
def test_effective_moduli_below_voigt(f):
    m = O.mask(32, f, 1)
    fv = m.mean()
    K, mu = O.effective_moduli(m, O.material())
    assert 0 < K < (1 - fv) * 5.0 and 0 < mu < (1 - fv) * 1.0
    # linear response: the strain amplitude does not matter
    K2, mu2 = O.effective_moduli(m, O.material(), strain=0.37)
    assert abs(K2 - K) < 1e-9 * K and abs(mu2 - mu) < 1e-9 * mu


def _ind(k, rng):
    e0 = np.cumsum(rng.uniform(0.05, 0.1, k))
    n = np.concatenate([[1.0, 1.0], np.linspace(0.9, 0.3, k - 2)])
    fp = np.linspace(0.0, 0.6, k)
    vmax = np.linspace(0.01, 0.4, k)
    ind = np.zeros((k, 8))
    ind[:, 0], ind[:, 2], ind[:, 3], ind[:, 5] = e0, fp, vmax, n
    L = 20
    st = np.zeros((k, 6), np.int32)
    st[:, 4] = (fp * 360).astype(np.int32)
    st[:, 5] = 40
    return ind, st, L


@pytest.mark.parametrize("load", ["equibiaxial", "shear"])
def test_empirical_curve_recovers_planted_alpha(load):
    """The fitted curve is A + alpha B with alpha the least-squares fit of
    sigma0; two fits of constant sigma0 expose A and B, and sigma0 planted
    as A + 0.37 B fits back alpha = 0.37 exactly.  A starts with the elastic
    slope: K~ eps0 (Eq. 5) or 2 mu~ eps0 (Eq. 6) at the first increment,
    where n = 1."""
    rng = np.random.default_rng(3)
    ind, st, L = _ind(12, rng)
    e = ind.copy()
    e[:, 1] = 1.0
    a1, f1 = O.empirical_curve(e, st, L, 2.5, load)
    e[:, 1] = 2.0
    a2, f2 = O.empirical_curve(e, st, L, 2.5, load)
    Bcol = (f2 - f1) / (a2 - a1)
    A = f1 - a1 * Bcol
    e[:, 1] = A + 0.37 * Bcol
    alpha, fit = O.empirical_curve(e, st, L, 2.5, load)
    assert abs(alpha - 0.37) < 1e-12
    np.testing.assert_allclose(fit, e[:, 1], atol=1e-12)
    slope = 2.5 if load == "equibiaxial" else 5.0
    assert abs(A[0] - slope * ind[0, 0]) < 1e-12


def test_eps_eq_closed_forms():
    g = 0.3
    assert abs(O.eps_eq(np.array([0.0, 0.0, 0.0, g])) - 2 * g / np.sqrt(3)) < 1e-15
    e = 0.2
    assert abs(O.eps_eq(np.array([e, 0.0, 0.0, 0.0])) - 2 * e / 3) < 1e-15
    assert O.eps_eq(np.array([0.1, 0.1, 0.1, 0.0])) < 1e-16  # hydrostatic: no deviator
