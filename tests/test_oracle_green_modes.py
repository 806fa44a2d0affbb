"""Pins of the oracle's other Green operators of Sec. 2 (CG1, DG1 and the
four operators of DG2) and of the CG2 average, against what the
mathematics fixes: the continuum operator is a real projector onto
compatible fields and the long-wavelength limit of Eq. 3; DG1 is real and
has the square symmetry of the grid; each DG2 operator at mirrored momenta
is exactly the mirror image of the Eq. 3 scheme on the mirrored lattice;
a mirror-symmetric problem gives a mirror-symmetric DG1 or DG2 solution and
an asymmetric Eq. 3 solution (Sec. 2)."""
import numpy as np
import pytest

import oracle as O

LAM0, MU0 = 1.5, 1.0
S = np.array([[[[(-1) ** (i + j + k + l) for l in range(2)] for k in range(2)] for j in range(2)] for i in range(2)])


def C0_apply(e, lam=LAM0, mu=MU0):
    return lam * np.trace(e) * np.eye(2) + 2 * mu * e


def G_apply(G, p):
    return np.einsum("ijkl,kl->ij", G, p)


def rand_sym(rng):
    a = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    return 0.5 * (a + a.T)


def qc(m, L):
    mm = m % L
    if mm > L // 2:
        mm -= L
    return 2 * np.pi * mm / L


FREQS = [(1, 0), (0, 1), (1, 1), (3, 5), (7, 2), (16, 3), (0, 16), (16, 16), (5, 27)]


@pytest.mark.parametrize("m1,m2", FREQS)
def test_cg1_is_real_symmetric_projector(m1, m2):
    """Real, with the minor and major symmetries; away from the Nyquist
    indices (where the sign of q_j = +-pi is ambiguous and the operator is
    the mean of both) a projector onto continuum-compatible fields."""
    L = 32
    G = O.green_mode(L, LAM0, MU0, O.GREEN_CG1, m1, m2)
    assert np.abs(G.imag).max() == 0.0
    g = G.real
    for perm in ("jikl", "ijlk", "klij"):
        np.testing.assert_allclose(np.einsum("ijkl->" + perm, g), g, atol=1e-15)
    if L // 2 in (m1, m2):
        return
    q = np.array([qc(m1, L), qc(m2, L)])
    rng = np.random.default_rng(m1 + 17 * m2)
    for _ in range(3):
        e = G_apply(G, rand_sym(rng))
        np.testing.assert_allclose(G_apply(G, C0_apply(e)), -e, atol=1e-13 * (1 + np.abs(e).max()))
        # continuum compatibility of the output: q2^2 e11 + q1^2 e22 - 2 q1 q2 e12 = 0
        assert abs(q[1] ** 2 * e[0, 0] + q[0] ** 2 * e[1, 1] - 2 * q[0] * q[1] * e[0, 1]) < 1e-13
        u = rng.standard_normal(2) + 1j * rng.standard_normal(2)
        ec = 0.5j * (np.outer(q, u) + np.outer(u, q))
        np.testing.assert_allclose(G_apply(G, C0_apply(ec)), -ec, atol=1e-13 * (1 + np.abs(ec).max()))


def test_cg1_is_even_in_q():
    L = 32
    for m1, m2 in FREQS:
        a = O.green_mode(L, LAM0, MU0, O.GREEN_CG1, m1, m2)
        b = O.green_mode(L, LAM0, MU0, O.GREEN_CG1, (L - m1) % L, (L - m2) % L)
        np.testing.assert_allclose(a, b, atol=1e-15)


@pytest.mark.parametrize("mode", [O.GREEN_CG1, O.GREEN_DG1])
def test_long_wavelength_limit_of_eq3(mode):
    """Sec. 2: the continuum operator is the long-wavelength limit of Eq. 3;
    the difference is first order in q (halves when q halves), and DG1 tends
    to the same limit."""
    L = 4096
    errs = []
    for m in (4, 2, 1):
        a = O.green(L, LAM0, MU0, m, 2 * m)
        b = O.green_mode(L, LAM0, MU0, mode, m, 2 * m)
        errs.append(np.abs(a - b).max() / np.abs(b).max())
    assert errs[2] < 2e-3
    assert 1.6 < errs[0] / errs[1] < 2.4 and 1.6 < errs[1] / errs[2] < 2.4


@pytest.mark.parametrize("m1,m2", FREQS)
def test_dg1_real_and_square_symmetric(m1, m2):
    """DG1 is real and respects the square symmetry of the grid: a mirror
    along x1 maps it to itself up to the tensor sign (-1)^(i+j+k+l), and so
    does the exchange x1 <-> x2 with indices 1 <-> 2."""
    L = 32
    G = O.green_mode(L, LAM0, MU0, O.GREEN_DG1, m1, m2)
    assert np.abs(G.imag).max() < 1e-16
    Gm = O.green_mode(L, LAM0, MU0, O.GREEN_DG1, (L - m1) % L, m2)
    np.testing.assert_allclose(Gm, S * G, atol=1e-15)
    Gs = O.green_mode(L, LAM0, MU0, O.GREEN_DG1, m2, m1)
    sw = np.array([1, 0])
    np.testing.assert_allclose(Gs[np.ix_(sw, sw, sw, sw)], G, atol=1e-15)
    # the plain Eq. 3 operator has neither property (the asymmetry of Sec. 2)
    G3 = O.green(L, LAM0, MU0, m1, m2)
    if m1 % 16 and m2 % 16:
        assert np.abs(O.green(L, LAM0, MU0, (L - m1) % L, m2) - S * G3).max() > 1e-3


def test_dg1_is_the_mean_of_the_dg2_operators():
    L = 32
    for m1, m2 in FREQS:
        G1 = O.green_mode(L, LAM0, MU0, O.GREEN_DG1, m1, m2)
        mem = [O.green_mode(L, LAM0, MU0, g, m1, m2) for g in O.DG2_MEMBERS]
        np.testing.assert_allclose(G1, np.mean(mem, axis=0), atol=1e-16)


@pytest.mark.parametrize("mode,axes", [(O.GREEN_EQ3_M1, (1,)), (O.GREEN_EQ3_M2, (2,)), (O.GREEN_EQ3_M12, (1, 2))])
def test_dg2_operator_is_the_mirrored_scheme(mode, axes):
    """An iteration with the operator at mirrored momenta equals, exactly, the
    mirror image of an Eq. 3 iteration on the mirrored lattice under the
    mirrored load (E12 and eps12 change sign with each mirror)."""
    L = 16
    mat = O.material()
    mask = O.mask(L, 0.2, 3)
    rng = np.random.default_rng(axes[0])
    E = np.array([0.4, 0.15, 0.0, 0.3])
    eps = E + 0.05 * rng.standard_normal((L, L, 4))
    a = O.al_step(mask, O.material(green=mode), E, eps)[0]
    b = O.al_step(O.mirror(mask, axes), mat, O.mirror_path(E, axes)[0], O.mirror(eps, axes))[0]
    np.testing.assert_allclose(a, O.mirror(b, axes), atol=1e-14)


def _symmetric_mask(L, f, seed, axes):
    m = O.mask(L, f, seed)
    for ax in axes:
        m = np.maximum(m, O.mirror(m, (ax,)))
    return m


def test_mirror_symmetric_problem_dg1_dg2_symmetric_eq3_not():
    """Sec. 2: Eq. 3 gives asymmetric field patterns; DG1 and DG2 restore the
    symmetry.  Mask symmetric under x1 -> -x1, equibiaxial load (mirror
    invariant)."""
    L = 16
    mask = _symmetric_mask(L, 0.15, 5, (1,))
    mat = O.material(Y=0.6)
    path = O.mirror_path(np.array([[0.2, 0.2, 0.0, 0.0], [0.4, 0.4, 0.0, 0.0]]), ())
    kw = dict(tol_eq=1e-9, tol_macro=1e-9, max_iter=3000)
    e3 = O.solve(mask, mat, path, **kw).eps
    d1 = O.solve(mask, O.material(Y=0.6, green=O.GREEN_DG1), path, **kw).eps
    d2 = O.solve_dg2(mask, mat, path, **kw).eps
    asym = lambda e: np.abs(e - O.mirror(e, (1,))).max() / np.abs(e).max()
    assert asym(e3) > 1e-3
    assert asym(d1) < 1e-12
    assert asym(d2) < 1e-12


def test_dg2_members_equal_mirrored_member_solves():
    """DG2's average is invariant under the mirrors: the DG2 field of the
    mirrored problem is the mirror image of the DG2 field (members permute)."""
    L = 8
    mask = O.mask(L, 0.2, 9)
    mat = O.material(Y=0.8)
    path = np.array([[0.0, 0.0, 0.0, 0.25], [0.0, 0.0, 0.0, 0.5]])
    kw = dict(tol_eq=1e-10, tol_macro=1e-10, max_iter=4000)
    a = O.solve_dg2(mask, mat, path, **kw)
    b = O.solve_dg2(O.mirror(mask, (1,)), mat, O.mirror_path(path, (1,)), **kw)
    np.testing.assert_allclose(O.mirror(b.eps, (1,)), a.eps, atol=1e-12)
    np.testing.assert_allclose(b.records["sig_mean"][:, :3], a.records["sig_mean"][:, :3], atol=1e-12)
    np.testing.assert_allclose(-b.records["sig_mean"][:, 3], a.records["sig_mean"][:, 3], atol=1e-12)


def test_cg1_homogeneous_closed_form():
    """f = 0: every operator gives the uniform solution eps = E (shear past
    the Mises limit: sigma12 = Y / sqrt(3))."""
    L = 8
    mask = np.zeros((L, L), np.uint8)
    g = 1.0 / (2 * np.sqrt(3))
    path = np.array([[0.0, 0.0, 0.0, 0.5 * g], [0.0, 0.0, 0.0, 2.0 * g]])
    for mode in (O.GREEN_CG1, O.GREEN_DG1):
        s = O.solve(mask, O.material(green=mode), path)
        assert s.status == 0
        np.testing.assert_allclose(s.records["sig_mean"][:, 3], [2 * 0.5 * g, 1 / np.sqrt(3)], rtol=1e-12)
        np.testing.assert_allclose(s.eps, np.broadcast_to(path[-1], (L, L, 4)), atol=1e-14)


def test_avg5_stencil():
    """CG2: a unit value at one pixel spreads as 1/5 over it and its four
    neighbours (periodic); constants are unchanged; the mean is kept."""
    L = 8
    f = np.zeros((L, L, 4))
    f[0, 0, 2] = 1.0
    g = O.avg5(f)
    exp = np.zeros((L, L))
    for x2, x1 in ((0, 0), (0, 1), (0, L - 1), (1, 0), (L - 1, 0)):
        exp[x2, x1] = 0.2
    np.testing.assert_allclose(g[..., 2], exp, atol=1e-16)
    assert np.abs(g[..., (0, 1, 3)]).max() == 0.0
    rng = np.random.default_rng(2)
    r = rng.standard_normal((L, L, 4))
    np.testing.assert_allclose(O.avg5(r).mean(axis=(0, 1)), r.mean(axis=(0, 1)), atol=1e-15)
    np.testing.assert_allclose(O.avg5(np.ones((L, L, 4)) * 3.0), 3.0, atol=1e-15)
