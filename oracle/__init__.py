"""Oracle: plain FP64 CPU reference of the augmented-Lagrangian FFT scheme with
the discrete Green operator (Willot & Pellegrini, arXiv:0802.2488, Sec. 2).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its binding) never imports this package, and this package
never imports the product.

This module compiles ``oracle.c`` with gcc into ``_liboracle.so`` (beside it)
and wraps it with ctypes and numpy.  Every function names the passage of the
paper it follows; the arithmetic itself lives in ``oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc, -O2, OpenMP, IEEE arithmetic) if stale."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(
                ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                 "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def threads() -> int:
    """OpenMP threads the oracle's loops use."""
    return int(lib().orc_threads())


def set_threads(n: int) -> None:
    """Sets the OpenMP threads of the oracle's loops (n > 0)."""
    lib().orc_set_threads(int(n))


class Material(C.Structure):
    """Matrix Lame moduli, Mises flow stress Y (inf = elastic), the
    reference medium C0 of the augmented Lagrangian and the Green operator
    (GREEN_* below)."""
    _fields_ = [("lambda_", C.c_double), ("mu", C.c_double), ("yield_", C.c_double),
                ("lambda0", C.c_double), ("mu0", C.c_double), ("green", C.c_int32),
                ("pad", C.c_int32)]


# Green operators of Sec. 2 (values of orc_material.green)
GREEN_EQ3, GREEN_CG1, GREEN_DG1, GREEN_EQ3_M1, GREEN_EQ3_M2, GREEN_EQ3_M12 = range(6)
# the four operators G(q1,q2), G(-q1,-q2), G(-q1,q2), G(q1,-q2) of DG2
DG2_MEMBERS = (GREEN_EQ3, GREEN_EQ3_M12, GREEN_EQ3_M1, GREEN_EQ3_M2)


class Control(C.Structure):
    _fields_ = [("tol_eq", C.c_double), ("tol_macro", C.c_double),
                ("max_iter", C.c_int32), ("eq_test", C.c_int32)]


# Equilibrium test (values of orc_control.eq_test): each operator's own
# (eta1 for Eq. 3, eta3 for CG1 and DG1), or eta3 for every operator
EQ_OWN, EQ_FIXED_POINT = 0, 1


class Record(C.Structure):
    _fields_ = [("sig_mean", C.c_double * 4), ("eps_mean", C.c_double * 4),
                ("eta1", C.c_double), ("eta2", C.c_double), ("eta3", C.c_double),
                ("iterations", C.c_int32), ("n_plastic", C.c_int32),
                ("n_clusters", C.c_int32), ("status", C.c_int32)]


def material(lam=1.5, mu=1.0, Y=1.0, lam0=None, mu0=None, green=GREEN_EQ3) -> Material:
    return Material(lam, mu, Y, lam if lam0 is None else lam0, mu if mu0 is None else mu0, int(green), 0)


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_U8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_VP = C.c_void_p


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.orc_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_splitmix64.restype = C.c_uint64
        L.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_void_threshold.restype = C.c_uint64
        L.orc_void_threshold.argtypes = [C.c_double]
        L.orc_mask.argtypes = [C.c_int, C.c_double, C.c_uint64, _U8]
        L.orc_fft2.argtypes = [_VP, C.c_int, C.c_int]
        L.orc_green.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, _D]
        L.orc_green_mode.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, _D]
        L.orc_green_apply.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, _D, _VP, _VP]
        L.orc_avg5.argtypes = [C.c_int, _D, _D]
        L.orc_displacement.argtypes = [C.c_int, _D, _D]
        L.orc_sigma_field.argtypes = [C.c_int64, _D, _U8, C.POINTER(Material), _D, _VP]
        L.orc_local_field.argtypes = [C.c_int64, _D, _U8, C.POINTER(Material), _D, _VP]
        L.orc_al_step.argtypes = [C.c_int, _U8, C.POINTER(Material), _D, _D, _D, _VP, _VP]
        L.orc_stats.argtypes = [C.c_int, _U8, C.POINTER(Material), _D, _D, _D,
                                C.POINTER(C.c_double), C.POINTER(C.c_int32), _VP]
        L.orc_void_plastic.restype = C.c_int32
        L.orc_void_plastic.argtypes = [C.c_int, _U8, _U8, _I32, _I32]
        L.orc_label.restype = C.c_int32
        L.orc_label.argtypes = [C.c_int, _U8, C.c_int, _I32]
        L.orc_solve.restype = C.c_int32
        L.orc_solve.argtypes = [C.c_int, _U8, C.POINTER(Material), C.POINTER(Control),
                                C.c_int, _D, C.POINTER(Record), _VP, _VP, _VP]
        _lib = L
    return _lib


def _check_L(L: int) -> None:
    if L < 2 or (L & (L - 1)) != 0:
        raise ValueError(f"lattice side {L} is not a power of two >= 2")


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------
# Sec. 2: random void pixels
# --------------------------------------------------------------------------

def splitmix64(seed: int, i: int) -> int:
    """i-th output of the SplitMix64 stream seeded with `seed`."""
    return int(lib().orc_splitmix64(seed & (2**64 - 1), i))


def void_threshold(f: float) -> int:
    return int(lib().orc_void_threshold(float(f)))


def mask(L: int, f: float, seed: int) -> np.ndarray:
    """uint8 (L, L), 1 = void: i.i.d. Bernoulli(f) pixels (Sec. 2)."""
    out = np.empty((L, L), dtype=np.uint8)
    lib().orc_mask(L, float(f), seed & (2**64 - 1), out)
    return out


# --------------------------------------------------------------------------
# FFT and the Green operator, Eqs. 2-3
# --------------------------------------------------------------------------

def fft2(a: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised 2D DFT with kernel exp(sign i q.x) (oracle's own FFT)."""
    b = np.ascontiguousarray(a, dtype=np.complex128).copy()
    L = b.shape[0]
    assert b.shape == (L, L)
    _check_L(L)
    lib().orc_fft2(_ptr(b), L, sign)
    return b


def green(L: int, lam0: float, mu0: float, m1: int, m2: int) -> np.ndarray:
    """G_ijkl(q) of Eq. 3 as a complex (2, 2, 2, 2) array."""
    g = np.zeros(32, dtype=np.float64)
    lib().orc_green(L, lam0, mu0, m1, m2, g)
    return g.view(np.complex128).reshape(2, 2, 2, 2)


def green_mode(L: int, lam0: float, mu0: float, mode: int, m1: int, m2: int) -> np.ndarray:
    """Green operator `mode` (GREEN_*; Sec. 2) at q = 2 pi (m1, m2) / L as a
    complex (2, 2, 2, 2) array."""
    g = np.zeros(32, dtype=np.float64)
    lib().orc_green_mode(L, lam0, mu0, int(mode), m1, m2, g)
    return g.view(np.complex128).reshape(2, 2, 2, 2)


def green_apply(L, lam0, mu0, E, phat, mode=GREEN_EQ3):
    """e^ = G p^ on a full (3, L, L) spectrum (11, 22, 12); e^(0) = L^2 E."""
    _check_L(L)
    ph = np.ascontiguousarray(phat, dtype=np.complex128)
    eh = np.empty_like(ph)
    lib().orc_green_apply(L, lam0, mu0, int(mode), np.ascontiguousarray(E, dtype=np.float64),
                          _ptr(ph), _ptr(eh))
    return eh


def avg5(field: np.ndarray) -> np.ndarray:
    """CG2 post-processing (Sec. 2): mean of each pixel and its four nearest
    neighbours (periodic) of an (L, L, 4) field."""
    f = np.ascontiguousarray(field, dtype=np.float64)
    out = np.empty_like(f)
    lib().orc_avg5(f.shape[0], f, out)
    return out


# --------------------------------------------------------------------------
# Constitutive law and the local step
# --------------------------------------------------------------------------

def sigma(eps: np.ndarray, void: np.ndarray, mat: Material):
    """sigma(eps) on (..., 4) arrays; returns (sigma, plastic_branch)."""
    e = np.ascontiguousarray(eps, dtype=np.float64)
    v = np.ascontiguousarray(np.broadcast_to(void, e.shape[:-1]), dtype=np.uint8)
    s = np.empty_like(e)
    pl = np.empty(v.shape, dtype=np.uint8)
    lib().orc_sigma_field(v.size, e, v, C.byref(mat), s, _ptr(pl))
    return s, pl


def local_solve(tau: np.ndarray, void: np.ndarray, mat: Material):
    """Solution of sigma(eps) + C0:eps = tau on (..., 4) arrays."""
    t = np.ascontiguousarray(tau, dtype=np.float64)
    v = np.ascontiguousarray(np.broadcast_to(void, t.shape[:-1]), dtype=np.uint8)
    e = np.empty_like(t)
    pl = np.empty(v.shape, dtype=np.uint8)
    lib().orc_local_field(v.size, t, v, C.byref(mat), e, _ptr(pl))
    return e, pl


# --------------------------------------------------------------------------
# The augmented-Lagrangian iteration and its indicators
# --------------------------------------------------------------------------

def al_step(mask_: np.ndarray, mat: Material, E, eps: np.ndarray, lam: np.ndarray | None = None):
    """One AL iteration from (eps, lam) (lam defaults to sigma(eps)).
    Returns (eps_new, lam_new, e, plastic) as (L, L, 4) / (L, L) arrays."""
    L = mask_.shape[0]
    _check_L(L)
    m = np.ascontiguousarray(mask_, dtype=np.uint8)
    ep = np.ascontiguousarray(eps, dtype=np.float64).copy()
    la = sigma(ep, m, mat)[0] if lam is None else np.ascontiguousarray(lam, dtype=np.float64).copy()
    e = np.empty_like(ep)
    pl = np.empty((L, L), dtype=np.uint8)
    lib().orc_al_step(L, m, C.byref(mat), np.ascontiguousarray(E, dtype=np.float64),
                      ep, la, _ptr(e), _ptr(pl))
    return ep, la, e, pl


@dataclass
class Stats:
    sig_mean: np.ndarray
    eps_mean: np.ndarray
    div2_mean: float
    n_plastic: int
    plastic: np.ndarray


def stats(mask_: np.ndarray, mat: Material, eps: np.ndarray) -> Stats:
    """Mean stress / strain, <|div sigma|^2> (backward differences, Eq. 1)
    and plastic pixels of sigma(eps) (Sec. 2 "Convergence issues", Sec. 3)."""
    L = mask_.shape[0]
    m = np.ascontiguousarray(mask_, dtype=np.uint8)
    sm = np.empty(4)
    em = np.empty(4)
    d2 = C.c_double()
    npl = C.c_int32()
    pl = np.empty((L, L), dtype=np.uint8)
    lib().orc_stats(L, m, C.byref(mat), np.ascontiguousarray(eps, dtype=np.float64),
                    sm, em, C.byref(d2), C.byref(npl), _ptr(pl))
    return Stats(sm, em, d2.value, npl.value, pl)


def label(flag: np.ndarray, periodic: bool = True):
    """Nearest-neighbour clusters (Sec. 3, Hoshen-Kopelman); label = smallest
    linear index of the cluster, -1 off the flag.  Returns (labels, count)."""
    f = np.ascontiguousarray(flag, dtype=np.uint8)
    L = f.shape[0]
    lab = np.empty((L, L), dtype=np.int32)
    n = lib().orc_label(L, f, 1 if periodic else 0, lab)
    return lab, int(n)


def void_plastic(mask_: np.ndarray, plastic: np.ndarray):
    """Sec. 3: clusters of the void-plastic phase, each void-free cluster
    connected to its nearest void.  Returns (labels, stats) with stats =
    (clusters, pixels of the largest, clusters without plastic pixels,
    clusters of the voids alone, plastic pixels, void pixels)."""
    m = np.ascontiguousarray(mask_, dtype=np.uint8)
    p = np.ascontiguousarray(plastic, dtype=np.uint8)
    L = m.shape[0]
    lab = np.empty((L, L), dtype=np.int32)
    st = np.zeros(6, dtype=np.int32)
    lib().orc_void_plastic(L, m, p, lab, st)
    return lab, st


def indicators(records: np.ndarray, stats: np.ndarray, L: int, load: str) -> np.ndarray:
    """Geometric indicators of Sec. 3 per increment, (n_inc, 8) columns:
    eps0, sigma0, f_p, v_max, i, n, r, -d2 sigma0 / d eps0^2.
      eps0, sigma0: <eps_m>, <sigma_m> (in-plane means (11 + 22) / 2) for
        equibiaxial loading, <eps_12>, <sigma_12> for shear;
      f_p = plastic pixels / matrix pixels (v_p / (1 - f));
      v_max = pixels of the largest void-plastic cluster / L^2;
      i = void-plastic clusters without plastic pixels / clusters of voids;
      n = void-plastic clusters / clusters of voids (its value at eps0 = 0);
      r = dn / d eps0 and -d2 sigma0 / d eps0^2 by second-order finite
        differences on the (possibly uneven) eps0 grid, one-sided at the
        ends (numpy.gradient).
    stats: (n_inc, 6) rows of void_plastic."""
    rec = np.asarray(records)
    st = np.asarray(stats, dtype=np.float64)
    if load == "equibiaxial":
        e0 = 0.5 * (rec["eps_mean"][:, 0] + rec["eps_mean"][:, 1])
        s0 = 0.5 * (rec["sig_mean"][:, 0] + rec["sig_mean"][:, 1])
    else:
        e0 = rec["eps_mean"][:, 3].copy()
        s0 = rec["sig_mean"][:, 3].copy()
    n_px = float(L * L)
    fp = st[:, 4] / (n_px - st[:, 5])
    vmax = st[:, 1] / n_px
    i = st[:, 2] / st[:, 3]
    n = st[:, 0] / st[:, 3]
    if len(e0) >= 2:
        r = np.gradient(n, e0)
        d2 = -np.gradient(np.gradient(s0, e0), e0)
    else:
        r = np.zeros_like(n)
        d2 = np.zeros_like(n)
    return np.stack([e0, s0, fp, vmax, i, n, r, d2], axis=1)


RECORD_DTYPE = np.dtype([("sig_mean", "f8", 4), ("eps_mean", "f8", 4), ("eta1", "f8"),
                         ("eta2", "f8"), ("eta3", "f8"), ("iterations", "i4"),
                         ("n_plastic", "i4"), ("n_clusters", "i4"), ("status", "i4")])
assert RECORD_DTYPE.itemsize == C.sizeof(Record)


@dataclass
class Solution:
    status: int
    records: np.ndarray          # RECORD_DTYPE, one per increment
    eps: np.ndarray              # (L, L, 4) final local strain
    plastic: np.ndarray | None   # (n_inc, L, L)
    labels: np.ndarray | None    # (n_inc, L, L)


def solve(mask_: np.ndarray, mat: Material, path: np.ndarray, tol_eq=1e-8, tol_macro=1e-8,
          max_iter=10000, fields=False, eq_test=EQ_OWN) -> Solution:
    """Strain-controlled loading by increments (Sec. 2) with the AL scheme;
    path is (n_inc, 4) prescribed mean strains (11, 22, 33, 12)."""
    L = mask_.shape[0]
    _check_L(L)
    m = np.ascontiguousarray(mask_, dtype=np.uint8)
    P = np.ascontiguousarray(path, dtype=np.float64).reshape(-1, 4)
    n_inc = P.shape[0]
    recs = (Record * n_inc)()
    eps = np.empty((L, L, 4))
    pl = np.empty((n_inc, L, L), dtype=np.uint8) if fields else None
    lab = np.empty((n_inc, L, L), dtype=np.int32) if fields else None
    st = lib().orc_solve(L, m, C.byref(mat), C.byref(Control(tol_eq, tol_macro, max_iter, int(eq_test))),
                         n_inc, P, recs, _ptr(eps), _ptr(pl), _ptr(lab))
    arr = np.frombuffer(bytes(recs), dtype=RECORD_DTYPE).copy()
    return Solution(int(st), arr, eps, pl, lab)


def mirror(a: np.ndarray, axes) -> np.ndarray:
    """Pixel mirror x_j -> -x_j (mod L) of an (L, L) or (L, L, 4) field for
    each lattice direction j in `axes` (1 = x1, the fast index; 2 = x2).  A
    tensor field (last axis of 4: 11, 22, 33, 12) also changes the sign of
    its 12 component once per mirrored direction."""
    L = a.shape[0]
    idx = (-np.arange(L)) % L
    b = a
    for j in axes:
        b = b[:, idx] if j == 1 else b[idx, :]
        if b.ndim == 3:
            b = b.copy()
            b[..., 3] = -b[..., 3]
    return np.ascontiguousarray(b)


def mirror_path(path: np.ndarray, axes) -> np.ndarray:
    """Prescribed mean strains of the mirrored problem (E12 changes sign once
    per mirrored direction)."""
    P = np.array(path, dtype=np.float64).reshape(-1, 4)
    if len(axes) % 2 == 1:
        P[:, 3] = -P[:, 3]
    return P


# lattice mirrors equivalent to the four operators of DG2, in DG2_MEMBERS
# order: G(q1,q2), G(-q1,-q2), G(-q1,q2), G(q1,-q2)
DG2_MIRRORS = ((), (1, 2), (1,), (2,))


@dataclass
class DG2Solution:
    members: list                # the four Solutions (of the mirrored problems), DG2_MIRRORS order
    records: np.ndarray          # RECORD_DTYPE: means of the members' macro values
    eps: np.ndarray              # (L, L, 4): mean of the four final strain fields


def solve_dg2(mask_: np.ndarray, mat: Material, path: np.ndarray, tol_eq=1e-8, tol_macro=1e-8,
              max_iter=10000, eq_test=EQ_OWN) -> DG2Solution:
    """DG2 (Sec. 2): four complete solves with G(q1,q2), G(-q1,-q2),
    G(-q1,q2), G(q1,-q2) in turn; the result is the average of the four
    converged strain fields.  The solve with G at mirrored momenta is the
    mirror image of the Eq. 3 solve of the mirrored lattice under the
    mirrored load (forward differences of Eq. 1 become backward ones), so
    each member runs Eq. 3 on a mirrored problem and its field is mirrored
    back; each member's indicators are then those of its own scheme.  Per
    increment the macroscopic stress and strain of the four are averaged
    (mirrored back: E12, sigma12 change sign with an odd mirror); the
    indicators are the largest of the four, the iteration counts their sum."""
    sols, fields = [], []
    for ax in DG2_MIRRORS:
        s = solve(mirror(mask_, ax), mat, mirror_path(path, ax), tol_eq, tol_macro, max_iter, eq_test=eq_test)
        sols.append(s)
        fields.append(mirror(s.eps, ax))
    rec = sols[0].records.copy()
    for f in ("sig_mean", "eps_mean"):
        vals = []
        for s, ax in zip(sols, DG2_MIRRORS):
            v = s.records[f].copy()
            if len(ax) % 2 == 1:
                v[:, 3] = -v[:, 3]
            vals.append(v)
        rec[f] = np.mean(vals, axis=0)
    for f in ("eta1", "eta2", "eta3", "status"):
        rec[f] = np.max([s.records[f] for s in sols], axis=0)
    rec["iterations"] = np.sum([s.records["iterations"] for s in sols], axis=0)
    return DG2Solution(sols, rec, np.mean(fields, axis=0))


# --------------------------------------------------------------------------
# Sec. 3: effective moduli, the empirical stress-strain formulas (Eqs. 5-6)
# and the equivalent strain of Fig. 1
# --------------------------------------------------------------------------

def effective_moduli(mask_: np.ndarray, mat: Material, strain: float = 1e-3, tol=1e-10, max_iter=20000):
    """Effective in-plane moduli of the porous lattice with the elastic matrix
    (Y = inf): K~ = <sigma_m> / <eps_m> under equibiaxial strain and
    mu~ = <sigma_12> / (2 <eps_12>) under shear, with sigma_m, eps_m the
    in-plane means (11 + 22) / 2 (the slopes of sigma0(eps0) in Eqs. 5-6 at
    small strain; the void-free matrix gives 2 (lambda + mu) and mu)."""
    el = Material(mat.lambda_, mat.mu, np.inf, mat.lambda0, mat.mu0, mat.green, 0)
    a = solve(mask_, el, np.array([[strain, strain, 0.0, 0.0]]), tol, tol, max_iter)
    b = solve(mask_, el, np.array([[0.0, 0.0, 0.0, strain]]), tol, tol, max_iter)
    K = (a.records["sig_mean"][0, 0] + a.records["sig_mean"][0, 1]) / (
        a.records["eps_mean"][0, 0] + a.records["eps_mean"][0, 1])
    mu = b.records["sig_mean"][0, 3] / (2.0 * b.records["eps_mean"][0, 3])
    return float(K), float(mu)


def empirical_curve(ind: np.ndarray, stats: np.ndarray, L: int, modulus: float, load: str):
    """Eqs. 5 (pressure) and 6 (shear): the stress-strain curve rebuilt from
    the geometric indicators, with the fitting number alpha chosen by least
    squares against the computed sigma0.  Returns (alpha, sigma0_fit).
      Eq. 5: sigma0 ~ K~ int_0^eps0 {(n - n_inf)/(1 - n_inf) + alpha (v_p - v_p^max)};
      Eq. 6: sigma0 ~ alpha f_p + 2 mu~ int_0^eps0 (n - n_inf)/(1 - n_inf).
    Readings: n_inf is n at the last increment; v_p is the volume fraction
    of the void-plastic phase (voids and plastic pixels) and v_p^max that of
    its largest cluster, v_max; the integrals are trapezoidal on the
    increments' eps0 with the integrand at eps0 = 0 equal to its value at the
    first increment (elastic: no plastic pixel yet)."""
    e0, s0, fp, vmax, n = ind[:, 0], ind[:, 1], ind[:, 2], ind[:, 3], ind[:, 5]
    st = np.asarray(stats, dtype=np.float64)
    vp = (st[:, 4] + st[:, 5]) / float(L * L)
    ninf = n[-1]
    g1 = (n - ninf) / (1.0 - ninf) if ninf != 1.0 else np.zeros_like(n)

    def cumint(g):
        x = np.concatenate([[0.0], e0])
        y = np.concatenate([[g[0]], g])
        return np.concatenate([[0.0], np.cumsum(0.5 * (y[1:] + y[:-1]) * np.diff(x))])[1:]

    I1 = cumint(g1)
    if load == "equibiaxial":
        A, Bv = modulus * I1, modulus * cumint(vp - vmax)
    else:
        A, Bv = 2.0 * modulus * I1, fp
    den = float(np.dot(Bv, Bv))
    alpha = float(np.dot(s0 - A, Bv) / den) if den > 0 else 0.0
    return alpha, A + alpha * Bv


def eps_eq(eps: np.ndarray) -> np.ndarray:
    """Equivalent strain of Fig. 1: [(2/3) e'_ij e'_ij]^(1/2), e' the 3D
    deviator of (11, 22, 33, 12), e'_12 counted twice."""
    e = np.asarray(eps, dtype=np.float64)
    m = (e[..., 0] + e[..., 1] + e[..., 2]) / 3.0
    d = (e[..., 0] - m) ** 2 + (e[..., 1] - m) ** 2 + (e[..., 2] - m) ** 2 + 2.0 * e[..., 3] ** 2
    return np.sqrt(2.0 / 3.0 * d)


def displacement(eps: np.ndarray) -> np.ndarray:
    """Displacement field (L, L, 2) of an in-plane strain field (L, L, 4) by
    the formula of Sec. 2 (u(q) from eps(q) with k^2 = k1^2 + k2^2, zero mean;
    at the two frequencies where k^2 vanishes the same relation is inverted
    with |k|^2, see oracle.c)."""
    e = np.ascontiguousarray(eps, dtype=np.float64)
    L = e.shape[0]
    assert e.shape == (L, L, 4)
    _check_L(L)
    u = np.empty((L, L, 2))
    lib().orc_displacement(L, e, u)
    return u
