"""Pins of the oracle's augmented-Lagrangian iteration and load stepping:
per-iteration invariants that hold to round-off (mean strain, compatibility
and equilibrium of Eq. 1 in real space, the multiplier identity), closed-form
homogeneous solutions, brute-force finite-difference solves of Eq. 1 on
small lattices, Parseval for the Fourier-space residual of Sec. 2, and
lattice symmetries."""
import json
import os

import numpy as np
import pytest
import scipy.optimize

import oracle as O
from paper_0802_2488_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
MAT = O.material(lam=1.5, mu=1.0, Y=1.0)

# arrays are indexed [x2, x1, c]; forward / backward differences along x1, x2
F1 = lambda a: np.roll(a, -1, axis=1) - a
F2 = lambda a: np.roll(a, -1, axis=0) - a
B1 = lambda a: a - np.roll(a, 1, axis=1)
B2 = lambda a: a - np.roll(a, 1, axis=0)


def backward_div(s):
    """Eq. 1: div_i = sum_j [s_ij(x) - s_ij(x - e^j)], s as (..., 4) fields."""
    return B1(s[..., 0]) + B2(s[..., 3]), B1(s[..., 3]) + B2(s[..., 1])


def c0(a, lam0=1.5, mu0=1.0):
    out = 2 * mu0 * a
    out[..., :3] += lam0 * a[..., :3].sum(-1, keepdims=True)
    return out


def test_one_iteration_invariants():
    L = 16
    m = O.mask(L, 0.25, 11)
    E = np.array([0.3, -0.1, 0.05, 0.4])
    eps0 = inputs.random_strain(L, E, 0.5, seed=5)
    lam0 = O.sigma(eps0, m, MAT)[0]
    eps1, lam1, e, pl = O.al_step(m, MAT, E, eps0, lam0)
    # <e> = E and e33 = E33
    np.testing.assert_allclose(e.reshape(-1, 4).mean(0), E, atol=1e-14)
    assert np.abs(e[..., 2] - E[2]).max() == 0.0  # generalized plane strain: q3 = 0
    # forward-difference compatibility: D2+D2+ e11 + D1+D1+ e22 - 2 D1+D2+ e12 = 0
    comp = F2(F2(e[..., 0])) + F1(F1(e[..., 1])) - 2 * F1(F2(e[..., 3]))
    assert np.abs(comp).max() < 1e-13
    # C0:e + p^n, p^n = lam^n - C0:eps^n, has zero backward divergence (Eq. 1)
    s = c0(e) + lam0 - c0(eps0)
    d1, d2 = backward_div(s)
    assert max(np.abs(d1).max(), np.abs(d2).max()) < 1e-13
    # the multiplier update reproduces the constitutive stress of the new strain
    np.testing.assert_allclose(lam1, O.sigma(eps1, m, MAT)[0], atol=1e-13)
    # and the voids carry none
    assert np.abs(lam1[m == 1]).max() < 1e-13
    # the same with a backward-difference stencil must fail (sign convention)
    comp_b = B2(B2(e[..., 0])) + B1(B1(e[..., 1])) - 2 * B1(B2(e[..., 3]))
    assert np.abs(comp_b).max() > 1e-3


def test_iterations_converge_to_equilibrium():
    L = 16
    m = O.mask(L, 0.15, 2)
    E = np.array([0.2, 0.2, 0.0, 0.0])
    eps = np.tile(E, (L, L, 1))
    lam = None
    eta = []
    for _ in range(1500):
        eps, lam, e, _ = O.al_step(m, MAT, E, eps, lam)
        st = O.stats(m, MAT, eps)
        s = st.sig_mean
        eta.append(np.sqrt(st.div2_mean / (s[0] ** 2 + s[1] ** 2 + 2 * s[3] ** 2)))
    assert eta[-1] < 1e-7 * eta[0]
    d1, d2 = backward_div(O.sigma(eps, m, MAT)[0])
    assert np.sqrt(np.mean(d1 ** 2 + d2 ** 2)) < 1e-7
    # compatibility residual eps - e vanishes too
    assert np.abs(eps - e).max() < 1e-6


def _golden(name):
    with open(os.path.join(HERE, "golden", name)) as fh:
        return json.load(fh)


@pytest.mark.parametrize("material", ["baseline", "paper"])
def test_homogeneous_lattice_closed_forms(material):
    """f = 0: uniform fields, one iteration per increment, macroscopic stress
    equal to the closed forms of tests/golden/homogeneous.json, yield exactly
    at the Mises limit."""
    g = _golden("homogeneous.json")[material]
    mat = O.material(lam=g["lambda"], mu=g["mu"], Y=g["Y"])
    L = 8
    m = np.zeros((L, L), np.uint8)
    for mode in ("equibiaxial", "shear"):
        cases = g[mode]
        path = np.array([c["E"] for c in cases])
        sol = O.solve(m, mat, path, tol_eq=1e-12, tol_macro=1e-12, max_iter=5, fields=True)
        assert sol.status == 0
        r = sol.records
        assert (r["iterations"] == 1).all()
        for k, c in enumerate(cases):
            np.testing.assert_allclose(r["sig_mean"][k], c["sigma"], rtol=1e-13, atol=1e-14)
            np.testing.assert_allclose(r["eps_mean"][k], c["E"], atol=1e-15)
            assert r["n_plastic"][k] == (L * L if c["plastic"] else 0)
            assert r["n_clusters"][k] == (1 if c["plastic"] else 0)
        # the final field is uniform
        assert np.abs(sol.eps - sol.eps[0, 0]).max() < 1e-15
    # a prescribed out-of-plane strain E33 is carried exactly (q3 = 0)
    E = np.array([[0.1, 0.2, 0.07, 0.05]])
    sol = O.solve(m, mat, E, tol_eq=1e-12, tol_macro=1e-12, max_iter=5)
    np.testing.assert_allclose(sol.eps.reshape(-1, 4), np.repeat(E, L * L, 0), atol=1e-15)
    np.testing.assert_allclose(sol.records["sig_mean"][0], O.sigma(E, 0, mat)[0][0], rtol=1e-14)


# ---------------------------------------------------------------------------
# brute force: the finite-difference problem of Eq. 1 solved in real space
# ---------------------------------------------------------------------------

def strain_operator(L):
    """Dense B: u (2 L^2, [u1 plane, u2 plane]) -> (eps11, eps22, eps12) planes
    by the forward differences of Eq. 1."""
    n = L * L
    I = np.eye(n).reshape(n, L, L)  # unit displacement at each pixel
    d1 = (np.roll(I, -1, axis=2) - I).reshape(n, n).T  # D1+ acting on a plane
    d2 = (np.roll(I, -1, axis=1) - I).reshape(n, n).T
    Z = np.zeros((n, n))
    return np.block([[d1, Z], [Z, d2], [0.5 * d2, 0.5 * d1]])


def voigt_stiffness(lam, mu):
    # energy = 1/2 v^T D v with v = (e11, e22, g12 = 2 e12), e33 = 0
    return np.array([[lam + 2 * mu, lam, 0], [lam, lam + 2 * mu, 0], [0, 0, mu]])


def test_brute_force_linear_porous():
    """Y = inf: minimise sum_x 1/2 eps:C(x):eps over periodic u (dense
    least squares); the stress field is unique and must equal the oracle's."""
    L = 8
    m = O.mask(L, 0.2, 4)
    E = np.array([0.1, -0.03, 0.0, 0.05])
    mat = O.material(lam=1.5, mu=1.0, Y=np.inf)
    B = strain_operator(L)
    n = L * L
    Dm = voigt_stiffness(1.5, 1.0)
    V = np.diag([1.0, 1.0, 2.0])  # (e11, e22, e12) -> Voigt
    K = np.zeros((2 * n, 2 * n))
    f = np.zeros(2 * n)
    Ev = V @ E[[0, 1, 3]]
    for x in range(n):
        if m.flat[x]:
            continue
        Bx = V @ B[[x, n + x, 2 * n + x], :]
        K += Bx.T @ Dm @ Bx
        f -= Bx.T @ Dm @ Ev
    u = np.linalg.lstsq(K, f, rcond=1e-12)[0]
    ev = (B @ u).reshape(3, n).T + E[[0, 1, 3]]
    eps_bf = np.zeros((n, 4))
    eps_bf[:, [0, 1, 3]] = ev
    sig_bf = O.sigma(eps_bf.reshape(L, L, 4), m, mat)[0]
    sol = O.solve(m, mat, E[None, :], tol_eq=1e-13, tol_macro=1e-13, max_iter=20000)
    assert sol.status == 0
    sig = O.sigma(sol.eps, m, mat)[0]
    scale = np.abs(sig_bf).max()
    assert np.abs(sig - sig_bf).max() < 1e-10 * scale
    # strain agrees on matrix pixels (voids' strain is not unique)
    assert np.abs((sol.eps - eps_bf.reshape(L, L, 4))[m == 0]).max() < 1e-9


def test_brute_force_plastic_porous():
    """Elastic-perfectly plastic matrix: minimise the deformation-theory
    energy sum_x w(E + eps(u)) (convex, C1) over u; compare stresses."""
    L = 8
    m = O.mask(L, 0.15, 9)
    E = np.array([0.45, 0.45, 0.0, 0.1])  # past first yield around the voids
    lam, mu, Y = 1.5, 1.0, 1.0
    K = lam + 2 * mu / 3
    sY = np.sqrt(2 / 3) * Y
    B = strain_operator(L)
    n = L * L
    matrix = (m.reshape(-1) == 0)

    def energy(u):
        e = (B @ u).reshape(3, n).T + E[[0, 1, 3]]
        tr = e[:, 0] + e[:, 1]
        d = np.stack([e[:, 0] - tr / 3, e[:, 1] - tr / 3, -tr / 3, e[:, 2]], 1)
        nd = np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2 + d[:, 2] ** 2 + 2 * d[:, 3] ** 2)
        el = 2 * mu * nd <= sY
        w = 0.5 * K * tr ** 2 + np.where(el, mu * nd ** 2, sY * nd - sY ** 2 / (4 * mu))
        g = np.where(el, 2 * mu, sY / np.maximum(nd, 1e-300))
        s11 = K * tr + g * d[:, 0]
        s22 = K * tr + g * d[:, 1]
        s12 = g * d[:, 3]
        W = np.sum(w * matrix)
        # dW/du = B^T (s11, s22, 2 s12) restricted to the matrix
        sv = np.concatenate([s11 * matrix, s22 * matrix, 2 * s12 * matrix])
        return W, B.T @ sv

    res = scipy.optimize.minimize(energy, np.zeros(2 * n), jac=True, method="L-BFGS-B",
                                  options={"maxiter": 200000, "maxcor": 50, "ftol": 1e-300, "gtol": 1e-13})
    u = res.x
    ev = (B @ u).reshape(3, n).T + E[[0, 1, 3]]
    eps_bf = np.zeros((n, 4))
    eps_bf[:, [0, 1, 3]] = ev
    sig_bf = O.sigma(eps_bf.reshape(L, L, 4), m, MAT)[0]
    sol = O.solve(m, MAT, E[None, :], tol_eq=1e-12, tol_macro=1e-12, max_iter=200000)
    sig = O.sigma(sol.eps, m, MAT)[0]
    assert O.stats(m, MAT, sol.eps).n_plastic > 0
    assert np.abs(sig - sig_bf).max() < 1e-6 * np.abs(sig_bf).max()


# ---------------------------------------------------------------------------
# the Fourier form of the residual and lattice symmetries
# ---------------------------------------------------------------------------

def test_residual_parseval():
    """Sec. 2 computes <|div sigma|^2> in Fourier space; with the forward
    kernel exp(-i q.x) the backward difference is multiplication by
    1 - exp(-i q_j), and Parseval makes both forms equal."""
    L = 32
    m = O.mask(L, 0.2, 1)
    eps = inputs.random_strain(L, [0.4, 0.2, 0.0, 0.1], 0.3, seed=2)
    st = O.stats(m, MAT, eps)
    sig = O.sigma(eps, m, MAT)[0]
    q = 2 * np.pi * np.arange(L) / L
    b1 = (1 - np.exp(-1j * q))[None, :]
    b2 = (1 - np.exp(-1j * q))[:, None]
    s11, s22, s12 = (np.fft.fft2(sig[..., c]) for c in (0, 1, 3))
    d1 = b1 * s11 + b2 * s12
    d2 = b1 * s12 + b2 * s22
    four = (np.abs(d1) ** 2 + np.abs(d2) ** 2).sum() / L ** 4
    np.testing.assert_allclose(st.div2_mean, four, rtol=1e-12)


def _run(m, E, iters, mat=MAT):
    L = m.shape[0]
    eps = np.tile(np.asarray(E, float), (L, L, 1))
    lam = None
    for _ in range(iters):
        eps, lam, _, _ = O.al_step(m, mat, E, eps, lam)
    return eps


def test_transpose_and_shift_symmetry():
    L = 16
    m = O.mask(L, 0.2, 3)
    E = np.array([0.5, 0.3, 0.0, 0.2])
    eps = _run(m, E, 60)
    # x1 <-> x2 exchanges the forward differences of Eq. 1 among themselves
    Et = E[[1, 0, 2, 3]]
    epst = _run(m.T.copy(), Et, 60)
    np.testing.assert_allclose(epst, eps.transpose(1, 0, 2)[..., [1, 0, 2, 3]], atol=1e-11)
    # cyclic shift
    ms = np.roll(m, (3, 5), axis=(0, 1))
    epss = _run(ms, E, 60)
    np.testing.assert_allclose(epss, np.roll(eps, (3, 5), axis=(0, 1)), atol=1e-11)


def test_single_mirror_is_not_a_symmetry():
    """Sec. 2: forward and backward directions are not equivalent, so the
    field of a mirrored medium is not the mirrored field."""
    L = 16
    m = O.mask(L, 0.2, 3)
    E = np.array([0.4, 0.4, 0.0, 0.0])
    eps = _run(m, E, 200)
    mm = m[:, ::-1].copy()
    epsm = _run(mm, E, 200)
    mirrored = eps[:, ::-1].copy()
    mirrored[..., 3] *= -1
    assert np.abs(epsm - mirrored).max() > 1e-3


def test_linearity_without_yield():
    L = 16
    m = O.mask(L, 0.2, 8)
    mat = O.material(lam=1.5, mu=1.0, Y=np.inf)
    E = np.array([0.2, -0.1, 0.0, 0.05])
    a = _run(m, E, 40, mat)
    b = _run(m, 3.0 * E, 40, mat)
    np.testing.assert_allclose(b, 3.0 * a, atol=1e-13)


def test_all_void_lattice_is_stress_free():
    L = 8
    m = np.ones((L, L), np.uint8)
    sol = O.solve(m, MAT, np.array([[0.1, 0.1, 0.0, 0.0]]), max_iter=10)
    assert sol.status == 0
    assert sol.records["iterations"][0] == 1
    assert np.all(sol.records["sig_mean"][0] == 0)
    assert sol.records["n_plastic"][0] == 0
