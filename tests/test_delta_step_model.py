"""The difference formulas of the defect-correction form's FP32 local step
(csrc/dcpass.cuh: delta_step), restated in numpy float32, against FP64
differences of the local step of the augmented Lagrangian and of the stress
of its solution (the matrix law of Sec. 2: Mises cap on 2 mu |dev eps| at
sqrt(2/3) Y; voids carry no stress).  The base points straddle the plastic
threshold, the increments range from 1e-1 to 1e-6 of it, so that branch
crossings (elastic -> plastic and back) are exercised.  The error must be
of FP32 size relative to the difference itself, and the branch decisions
must match FP64's: that is what lets the form reach FP64 tolerances.
"""
import numpy as np
import pytest

import oracle as O

f32 = np.float32
MAT = O.material()  # mu = 1, lambda = 1.5, Y = 1, C0 = matrix
mu, lam, Y, mu0, lam0 = MAT.mu, MAT.lambda_, MAT.yield_, MAT.mu0, MAT.lambda0
K = lam + 2 * mu / 3
K0 = lam0 + 2 * mu0 / 3
ylim = np.sqrt(2 / 3) * Y
Tstar = ylim * (mu + mu0) / mu  # |tau'| where the local step turns plastic


def dev(a):
    m = (a[..., 0] + a[..., 1] + a[..., 2]) / 3
    d = a.copy()
    d[..., :3] -= m[..., None]
    return d, m


def nrm2(d):
    return d[..., 0] ** 2 + d[..., 1] ** 2 + d[..., 2] ** 2 + 2 * d[..., 3] ** 2


def LS64(t, void):
    """The oracle's local step and the stress of its solution (FP64)."""
    e, _ = O.local_solve(t, void.astype(np.uint8), MAT)
    s, pl = O.sigma(e, void.astype(np.uint8), MAT)
    return e, s, pl.astype(bool)


def delta32(tdev, h, dt_full, void):
    """tdev: base deviator (4, float32); h = |t|^2 - T*^2 (float32, exact-ish);
    dt_full: increment of tau (float32).  Returns d_eps, d_sig (float32)."""
    dd, dm = dev(dt_full)
    dd = dd.astype(f32); dm = dm.astype(f32)
    t = tdev.astype(f32)
    dem = np.where(void, dm / f32(3 * K0), dm / f32(3 * (K + K0))).astype(f32)
    # |t + dt|^2 - T*^2 = h + 2 t.dt + |dt|^2
    tdt = (t[..., 0]*dd[..., 0] + t[..., 1]*dd[..., 1] + t[..., 2]*dd[..., 2] + f32(2)*t[..., 3]*dd[..., 3]).astype(f32)
    dd2 = nrm2(dd).astype(f32)
    hb = (h + f32(2) * tdt + dd2).astype(f32)
    a2 = (h + f32(Tstar**2)).astype(f32)  # |t|^2
    b2 = (a2 + f32(2) * tdt + dd2).astype(f32)
    a = np.sqrt(a2).astype(f32); b = np.sqrt(b2).astype(f32)
    pa = (~void) & (h > 0); pb = (~void) & (hb > 0)
    # unit-vector difference n(t+dt) - n(t) = dt/b - t (2 t.dt + |dt|^2) / (a b (a + b))
    with np.errstate(divide="ignore", invalid="ignore"):
        dn = dd / b[..., None] - t * ((f32(2)*tdt + dd2) / (a * b * (a + b)))[..., None]
        nb = (t + dd) / b[..., None]
        # J(s) = n(s) (|s| mu/(mu+mu0) - ylim) / (2 mu0), |s| - T* = (|s|^2 - T*^2)/(|s| + T*)
        Jb = nb * ((f32(mu / (mu + mu0)) * hb / (b + f32(Tstar))) / f32(2 * mu0))[..., None]
    ce = f32(1 / (2 * (mu + mu0))); cp = f32(1 / (2 * mu0)); ry = f32(ylim / (2 * mu0))
    ge = f32(mu / (mu + mu0))
    de_EE = dd * ce; ds_EE = dd * ge
    de_PP = dd * cp - ry * dn; ds_PP = f32(ylim) * dn
    de_EP = dd * ce + Jb; ds_EP = dd * ge - f32(2 * mu0) * Jb
    de_PE = de_PP - Jb; ds_PE = ds_PP + f32(2 * mu0) * Jb
    de_V = dd * cp; ds_V = np.zeros_like(dd)
    sel = lambda ee, pp, ep, pe, vv: np.where(void[..., None], vv, np.where((pa & pb)[..., None], pp, np.where((~pa & ~pb)[..., None], ee, np.where(pb[..., None], ep, pe))))
    de = sel(de_EE, de_PP, de_EP, de_PE, de_V)
    ds = sel(ds_EE, ds_PP, ds_EP, ds_PE, ds_V)
    de = de.copy(); de[..., :3] += dem[..., None]
    ds = ds.copy(); ds[..., :3] += np.where(void, f32(0), f32(3 * K) * dem)[..., None]
    return de.astype(f32), ds.astype(f32), pb



@pytest.mark.parametrize("mag", [1e-1, 1e-3, 1e-6])
def test_delta_step_is_accurate_relative_to_the_difference(mag):
    rng = np.random.default_rng(0)
    N = 40000
    void = rng.random(N) < 0.1
    t = rng.standard_normal((N, 4))
    t[:, 2] = rng.standard_normal(N) * 0.3
    tdv, tm = dev(t)
    r = np.sqrt(nrm2(tdv))
    t = t * (Tstar * np.exp(rng.uniform(-0.5, 0.5, N)) / r)[:, None]
    dt = rng.standard_normal((N, 4)) * mag
    e0, s0, p0 = LS64(t, void)
    e1, s1, p1 = LS64(t + dt, void)
    tdev, _ = dev(t)
    h = (nrm2(tdev) - Tstar ** 2).astype(f32)
    de, ds, pb = delta32(tdev, h, dt.astype(f32), void)
    ref_de, ref_ds = e1 - e0, s1 - s0
    scale = np.abs(dt).max(axis=1)
    err_e = np.abs(de - ref_de).max(axis=1) / scale
    err_s = np.abs(ds - ref_ds).max(axis=1) / scale
    assert (pb == p1).all()
    assert err_e.max() < 2e-6 and err_s.max() < 2e-5, (err_e.max(), err_s.max())
    if mag >= 1e-3:
        assert ((p0 != p1) & ~void).sum() > 10  # threshold crossings were exercised
