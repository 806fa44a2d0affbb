"""Pins of the oracle's constitutive law and local step: the Mises cap
sigma_eq <= Y with equality on the plastic zone (Sec. 2-3), Hooke's law in
Lame form below yield, zero stress in voids, and the defining equation
sigma(eps) + C0:eps = tau of the augmented-Lagrangian local step."""
import numpy as np

import oracle as O

MAT = O.material(lam=1.5, mu=1.0, Y=1.0)


def full(t):
    """(..., 4) (11,22,33,12) -> (..., 3, 3)."""
    a = np.zeros(t.shape[:-1] + (3, 3))
    a[..., 0, 0], a[..., 1, 1], a[..., 2, 2] = t[..., 0], t[..., 1], t[..., 2]
    a[..., 0, 1] = a[..., 1, 0] = t[..., 3]
    return a


def mises(sig):
    s = full(sig)
    dev = s - np.trace(s, axis1=-2, axis2=-1)[..., None, None] / 3 * np.eye(3)
    return np.sqrt(1.5 * np.einsum("...ij,...ij->...", dev, dev))


def test_elastic_branch_is_hooke_lame_form():
    rng = np.random.default_rng(0)
    eps = 0.05 * rng.uniform(-1, 1, size=(500, 4))
    sig, pl = O.sigma(eps, 0, MAT)
    assert not pl.any()
    e = full(eps)
    ref = 1.5 * np.trace(e, axis1=1, axis2=2)[:, None, None] * np.eye(3) + 2.0 * e
    np.testing.assert_allclose(full(sig), ref, atol=1e-14)


def test_mises_cap_and_plastic_zone():
    rng = np.random.default_rng(1)
    eps = rng.uniform(-2, 2, size=(2000, 4)) * rng.uniform(0, 1, size=(2000, 1)) ** 3
    sig, pl = O.sigma(eps, 0, MAT)
    se = mises(sig)
    assert pl.sum() > 100 and (pl == 0).sum() > 100
    assert (se <= 1.0 + 1e-13).all()
    np.testing.assert_allclose(se[pl == 1], 1.0, rtol=1e-14)
    assert (se[pl == 0] <= 1.0).all()
    # mean stress = K tr(eps) on both branches; stress deviator parallel to
    # the strain deviator
    K = 1.5 + 2.0 / 3.0
    s, e = full(sig), full(eps)
    np.testing.assert_allclose(np.trace(s, axis1=1, axis2=2) / 3, K * np.trace(e, axis1=1, axis2=2), atol=1e-12)
    sd = s - np.trace(s, axis1=1, axis2=2)[:, None, None] / 3 * np.eye(3)
    ed = e - np.trace(e, axis1=1, axis2=2)[:, None, None] / 3 * np.eye(3)
    cross = np.einsum("nij,nij->n", sd, ed) ** 2 - np.einsum("nij,nij->n", sd, sd) * np.einsum("nij,nij->n", ed, ed)
    assert np.abs(cross).max() < 1e-10


def test_void_pixels_carry_no_stress():
    rng = np.random.default_rng(2)
    eps = rng.uniform(-3, 3, size=(100, 4))
    sig, pl = O.sigma(eps, 1, MAT)
    assert (sig == 0).all() and not pl.any()


def test_local_step_solves_its_equation():
    """eps = local(tau) must satisfy sigma(eps) + C0:eps = tau, on both branches
    of the matrix and in voids, for several reference media."""
    rng = np.random.default_rng(3)
    for lam0, mu0 in [(1.5, 1.0), (0.75, 0.5), (3.0, 2.0)]:
        mat = O.material(lam=1.5, mu=1.0, Y=1.0, lam0=lam0, mu0=mu0)
        tau = rng.uniform(-6, 6, size=(3000, 4))
        void = (rng.random(3000) < 0.3).astype(np.uint8)
        eps, pl = O.local_solve(tau, void, mat)
        sig, pl2 = O.sigma(eps, void, mat)
        tr = eps[:, :3].sum(1)
        c0 = np.empty_like(eps)
        c0[:, :3] = lam0 * tr[:, None] + 2 * mu0 * eps[:, :3]
        c0[:, 3] = 2 * mu0 * eps[:, 3]
        np.testing.assert_allclose(sig + c0, tau, atol=1e-12)
        assert pl.sum() > 100
        # the branch of the local step is the branch of sigma at its solution
        # (equal except at pixels numerically on the yield surface)
        assert (pl != pl2).sum() <= 2


def test_local_step_is_continuous_across_yield():
    mat = MAT
    d = np.array([1.0, -0.5, -0.5, 0.3])
    d = d / np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2 + 2 * d[3] ** 2)
    # elastic trial |dev| = |tau'| / (2 (mu + mu0)) reaches sqrt(2/3) Y / (2 mu) at
    # |tau'| = sqrt(2/3) * (mu + mu0) / mu
    t0 = np.sqrt(2 / 3) * 2.0
    ts = t0 * (1 + np.array([-1e-9, 1e-9]))
    tau = ts[:, None] * d[None, :] + np.array([0.3, 0.3, 0.3, 0.0])
    eps, pl = O.local_solve(tau, 0, mat)
    assert pl.tolist() == [0, 1]
    assert np.abs(eps[0] - eps[1]).max() < 1e-8
