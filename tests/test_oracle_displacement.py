"""Pins of the oracle's displacement field (Sec. 2): a displacement differenced
in real space with the forward differences of Eq. 1 comes back exactly
(minus its mean, the irrelevant mode q = 0), also through the frequencies
where k1^2 + k2^2 vanishes; shifts commute; a uniform strain has no
periodic displacement."""
import numpy as np
import pytest

import oracle as O


def strain_of(u):
    """Forward-difference strain (L, L, 4) of a periodic displacement
    (L, L, 2) at [x2][x1]: e11 = D1 u1, e22 = D2 u2, e12 = (D2 u1 + D1 u2)/2,
    D_j f(x) = f(x + e_j) - f(x); e33 = 0."""
    u1, u2 = u[..., 0], u[..., 1]
    d1 = lambda f: np.roll(f, -1, axis=1) - f
    d2 = lambda f: np.roll(f, -1, axis=0) - f
    e = np.zeros(u.shape[:2] + (4,))
    e[..., 0] = d1(u1)
    e[..., 1] = d2(u2)
    e[..., 3] = 0.5 * (d2(u1) + d1(u2))
    return e


@pytest.mark.parametrize("L", [4, 8, 16, 64, 128])
def test_forward_difference_round_trip(L):
    rng = np.random.default_rng(L)
    u = rng.standard_normal((L, L, 2))
    got = O.displacement(strain_of(u))
    ref = u - u.mean(axis=(0, 1))
    np.testing.assert_allclose(got, ref, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("L", [8, 32])
@pytest.mark.parametrize("m", [(1, 3), (3, 1)])
def test_mode_where_k_squared_vanishes(L, m):
    """u of one Fourier mode at q = (pi/2, 3pi/2) or (3pi/2, pi/2), where the
    formula's denominator k1^2 + k2^2 is zero."""
    m1, m2 = m[0] * L // 4, m[1] * L // 4
    x2, x1 = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    ph = 2 * np.pi * (m1 * x1 + m2 * x2) / L
    u = np.stack([np.cos(ph) + 0.3 * np.sin(ph), -0.7 * np.cos(ph + 0.4)], axis=-1)
    got = O.displacement(strain_of(u))
    np.testing.assert_allclose(got, u - u.mean(axis=(0, 1)), atol=1e-13)


def test_shift_commutes():
    L = 16
    rng = np.random.default_rng(1)
    e = rng.standard_normal((L, L, 4))
    a = O.displacement(np.roll(e, (3, -5), axis=(0, 1)))
    b = np.roll(O.displacement(e), (3, -5), axis=(0, 1))
    np.testing.assert_allclose(a, b, atol=1e-13)


def test_uniform_strain_has_no_periodic_displacement():
    L = 8
    e = np.broadcast_to(np.array([0.3, -0.1, 0.0, 0.2]), (L, L, 4)).copy()
    assert np.abs(O.displacement(e)).max() < 1e-15
