"""Pins of the oracle's FFT and discrete Green operator (Eqs. 1-3) against
what the mathematics fixes: a library FFT, the projector and equilibrium
properties that define a Green operator, the symmetries stated in Sec. 2,
and the continuum limit (textbook Moulinec-Suquet operator)."""
import numpy as np
import pytest

import oracle as O

LAM0, MU0 = 1.5, 1.0


def C0_apply(e, lam=LAM0, mu=MU0):
    """Isotropic stiffness on a 2x2 (in-plane, plane-strain) complex tensor."""
    return lam * np.trace(e) * np.eye(2) + 2 * mu * e


def eq2_k(m, L):
    # Fourier symbol of the forward difference u(x+e_j) - u(x) = i k_j u^ under
    # the forward kernel exp(-i q.x): i k_j = exp(i q_j) - 1.
    q = 2 * np.pi * m / L
    return (np.exp(1j * q) - 1) / 1j


def rand_sym(rng):
    a = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    return 0.5 * (a + a.T)


def G_apply(G, p):
    return np.einsum("ijkl,kl->ij", G, p)


@pytest.mark.parametrize("L", [4, 8, 16, 64])
def test_fft_matches_library(L):
    rng = np.random.default_rng(L)
    a = rng.standard_normal((L, L)) + 1j * rng.standard_normal((L, L))
    np.testing.assert_allclose(O.fft2(a, -1), np.fft.fft2(a), rtol=0, atol=1e-11 * L * L)
    np.testing.assert_allclose(O.fft2(a, +1), np.fft.ifft2(a) * L * L, rtol=0, atol=1e-11 * L * L)


def test_k_symbol_is_eq2():
    # Eq. 2 states k_j = 2 sin(q_j/2) exp(i q_j/2); the forward-difference symbol
    # above must be the same number (this fixes the DFT sign convention).
    for L in (8, 64):
        for m in range(L):
            q = 2 * np.pi * m / L
            assert abs(eq2_k(m, L) - 2 * np.sin(q / 2) * np.exp(1j * q / 2)) < 1e-14


FREQS = [(1, 0), (0, 1), (1, 1), (3, 5), (7, 2), (8, 8), (15, 1), (5, 13), (16, 3), (0, 16), (16, 16)]


@pytest.mark.parametrize("m1,m2", FREQS)
def test_green_solves_equilibrium_and_compatibility(m1, m2):
    """e^ = G p^ must be (a) compatible: e^ = sym(i k (x) u) for some u, and
    (b) make C0:e^ + p^ equilibrated: i k*_l (C0 e^ + p^)_kl = 0 (Eq. 2)."""
    L = 32
    G = O.green(L, LAM0, MU0, m1, m2)
    k = np.array([eq2_k(m1, L), eq2_k(m2, L)])
    rng = np.random.default_rng(m1 * 100 + m2)
    for _ in range(4):
        p = rand_sym(rng)
        e = G_apply(G, p)
        # compatibility in 2D: k2^2 e11 + k1^2 e22 - 2 k1 k2 e12 = 0
        comp = k[1] ** 2 * e[0, 0] + k[0] ** 2 * e[1, 1] - 2 * k[0] * k[1] * e[0, 1]
        assert abs(comp) < 1e-13 * (1 + np.abs(p).max())
        s = C0_apply(e) + p
        div = 1j * np.conj(k) @ s  # i k*_l s_kl, indexed by k (s symmetric)
        assert np.abs(div).max() < 1e-13 * (1 + np.abs(p).max())
        assert abs(e[0, 1] - e[1, 0]) < 1e-15 * (1 + np.abs(p).max())


@pytest.mark.parametrize("m1,m2", FREQS)
def test_green_is_projector(m1, m2):
    """G C0 G = -G (i.e. Gamma0 C0 Gamma0 = Gamma0 with Gamma0 = -G), and
    G C0 eps_c = -eps_c for a compatible strain eps_c = sym(i k (x) u)."""
    L = 32
    G = O.green(L, LAM0, MU0, m1, m2)
    k = np.array([eq2_k(m1, L), eq2_k(m2, L)])
    rng = np.random.default_rng(7 + m1 + 31 * m2)
    for _ in range(4):
        p = rand_sym(rng)
        e = G_apply(G, p)
        np.testing.assert_allclose(G_apply(G, C0_apply(e)), -e, atol=1e-13 * (1 + np.abs(e).max()))
        u = rng.standard_normal(2) + 1j * rng.standard_normal(2)
        ec = 0.5j * (np.outer(k, u) + np.outer(u, k))
        np.testing.assert_allclose(G_apply(G, C0_apply(ec)), -ec, atol=1e-13 * (1 + np.abs(ec).max()))


def test_green_annihilates_equilibrated_stress():
    """A stress field with zero backward-difference divergence (Eq. 1), built
    in real space from a stress function, has G sigma^ = 0 at every q."""
    L = 16
    rng = np.random.default_rng(3)
    phi = rng.standard_normal((L, L))
    # arrays indexed [x2, x1]; backward differences D1-, D2-
    D1 = lambda a: a - np.roll(a, 1, axis=1)
    D2 = lambda a: a - np.roll(a, 1, axis=0)
    s11, s22, s12 = D2(D2(phi)), D1(D1(phi)), -D1(D2(phi))
    # real-space check that it is equilibrated in the sense of Eq. 1
    assert np.abs(D1(s11) + D2(s12)).max() < 1e-12
    assert np.abs(D1(s12) + D2(s22)).max() < 1e-12
    sh = np.stack([np.fft.fft2(s) for s in (s11, s22, s12)])
    eh = O.green_apply(L, LAM0, MU0, np.zeros(4), sh)
    eh[:, 0, 0] = 0
    assert np.abs(eh).max() < 1e-11 * np.abs(sh).max()


def test_green_zero_frequency_and_symmetries():
    L = 32
    assert np.abs(O.green(L, LAM0, MU0, 0, 0)).max() == 0.0
    for m1, m2 in FREQS:
        G = O.green(L, LAM0, MU0, m1, m2)
        Gm = O.green(L, LAM0, MU0, (L - m1) % L, (L - m2) % L)
        # real fields stay real: G(-q) = G(q)*
        np.testing.assert_allclose(Gm, np.conj(G), atol=1e-14)
        # Sec. 2: G_ijkl = G*_klij, and minor symmetries
        np.testing.assert_allclose(G, np.conj(G.transpose(2, 3, 0, 1)), atol=1e-14)
        np.testing.assert_allclose(G, G.transpose(1, 0, 2, 3), atol=1e-15)
        np.testing.assert_allclose(G, G.transpose(0, 1, 3, 2), atol=1e-15)
    # Sec. 2: nonzero imaginary part, hence no major symmetry, off the axes
    G = O.green(L, LAM0, MU0, 3, 5)
    assert np.abs(G.imag).max() > 1e-3
    assert np.abs(G - G.transpose(2, 3, 0, 1)).max() > 1e-3


def continuum_gamma0(xi, lam0, mu0):
    """Textbook isotropic Green operator of the strain (Moulinec-Suquet):
    Gamma0_ijkl = [d_ki x_l x_j + d_li x_k x_j + d_kj x_l x_i + d_lj x_k x_i] / (4 mu0 |x|^2)
                  - (lam0 + mu0) / (mu0 (lam0 + 2 mu0)) x_i x_j x_k x_l / |x|^4."""
    d = np.eye(2)
    n2 = xi @ xi
    g = (np.einsum("ki,l,j->ijkl", d, xi, xi) + np.einsum("li,k,j->ijkl", d, xi, xi)
         + np.einsum("kj,l,i->ijkl", d, xi, xi) + np.einsum("lj,k,i->ijkl", d, xi, xi)) / (4 * mu0 * n2)
    g -= (lam0 + mu0) / (mu0 * (lam0 + 2 * mu0)) * np.einsum("i,j,k,l->ijkl", xi, xi, xi, xi) / n2 ** 2
    return g


def test_green_continuum_limit():
    """Sec. 2: the continuum Green operator is retrieved for q1, q2 << 1;
    here G = -Gamma0 and the deviation is O(|q|)."""
    L = 4096
    for (m1, m2) in [(1, 0), (1, 1), (2, 3), (5, 1)]:
        q = 2 * np.pi * np.array([m1, m2]) / L
        G = O.green(L, LAM0, MU0, m1, m2)
        Gc = -continuum_gamma0(q, LAM0, MU0)
        err = np.abs(G - Gc).max() / np.abs(Gc).max()
        assert err < 2 * np.linalg.norm(q), (m1, m2, err)
    # and it is not the continuum operator at large q
    G = O.green(64, LAM0, MU0, 16, 8)
    q = 2 * np.pi * np.array([16, 8]) / 64
    assert np.abs(G - (-continuum_gamma0(q, LAM0, MU0))).max() > 1e-2
