"""Thin ctypes binding of libepfft.so (include/epfft.h): argument marshalling
only, every step of the computation runs in the library's CUDA kernels.

The functions keep the C names.  Device memory is torch's: the context
allocates through torch's caching allocator (the C ABI's allocator hook),
device-side inputs and outputs are torch CUDA tensors, and host-side ones are
numpy arrays.  There is no fallback: if the library is missing or cannot be
loaded every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libepfft.so")

EPFFT_OK = 0
EPFFT_PENDING = 1
EPFFT_ERR_ARG = -1
EPFFT_ERR_OOM = -2
EPFFT_ERR_NUMERIC = -3
EPFFT_NOT_CONVERGED = -4
EPFFT_ERR_DEVICE_TIMEOUT = -5
EPFFT_ERR_CUDA = -6
EPFFT_ERR_UNSUPPORTED = -7
EPFFT_ERR_SCRATCH_LIMIT = -8
N_TILINGS = 4  # EPFFT_N_TILINGS
EPFFT_FP64 = 0
EPFFT_FP32 = 1
EPFFT_FP32_DEFECT = 2
# 'fp32_defect': FP64 state with FP32 transforms of the polarization's
# difference from an FP64-transformed reference (defect correction)
_PREC = {"fp64": EPFFT_FP64, "fp32": EPFFT_FP32, "fp32_defect": EPFFT_FP32_DEFECT}
EPFFT_GREEN_EQ3 = 0
EPFFT_GREEN_CG1 = 1
EPFFT_GREEN_DG1 = 2
_GREEN = {"eq3": EPFFT_GREEN_EQ3, "cg1": EPFFT_GREEN_CG1, "dg1": EPFFT_GREEN_DG1}
EPFFT_WANT_EPS = 1
EPFFT_WANT_SIG = 2
EPFFT_WANT_PLASTIC = 4
EPFFT_WANT_LABELS = 8
EPFFT_EQ_OWN = 0
EPFFT_EQ_FIXED_POINT = 1
_EQ_TEST = {"own": EPFFT_EQ_OWN, "fixed_point": EPFFT_EQ_FIXED_POINT}

SYMBOLS = ["epfft_create", "epfft_destroy", "epfft_last_stats", "epfft_strerror", "epfft_supported",
           "epfft_solve", "epfft_solve_batch", "epfft_mask", "epfft_iterate", "epfft_project", "epfft_label",
           "epfft_time_passes", "epfft_project_static", "epfft_serve_open", "epfft_serve_close",
           "epfft_submit", "epfft_serve_step", "epfft_poll", "epfft_autotune", "epfft_set_tiling",
           "epfft_solve_dg2", "epfft_average5", "epfft_void_plastic", "epfft_indicators",
           "epfft_effective_moduli", "epfft_empirical_curve", "epfft_eps_eq", "epfft_displacement",
           "epfft_ticket_fields", "epfft_release", "epfft_solve_refined", "epfft_solve_refined_batch",
           "epfft_fp64_peak", "epfft_supported_tiling", "epfft_set_defect_refresh"]


class EpfftError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


AllocFn = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FreeFn = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class _Options(C.Structure):
    _fields_ = [("device", C.c_int32), ("reserved", C.c_int32), ("stream", C.c_void_p),
                ("alloc", AllocFn), ("free", FreeFn), ("alloc_user", C.c_void_p)]


class _Problem(C.Structure):
    _fields_ = [("L", C.c_int32), ("precision", C.c_int32), ("void_fraction", C.c_double),
                ("seed", C.c_uint64), ("mask", C.c_void_p), ("mask_on_device", C.c_int32),
                ("green", C.c_int32), ("mu", C.c_double), ("lambda_", C.c_double),
                ("yield_stress", C.c_double), ("mu0", C.c_double), ("lambda0", C.c_double),
                ("tol_eq", C.c_double), ("tol_macro", C.c_double), ("max_iter", C.c_int32),
                ("eq_test", C.c_int32)]


class _Path(C.Structure):
    _fields_ = [("n_inc", C.c_int32), ("reserved", C.c_int32), ("E", C.c_void_p)]


class _Stats(C.Structure):
    _fields_ = [("loop_steps", C.c_int64), ("kernel_launches", C.c_int64), ("iterations", C.c_int64)]


class _ServeOptions(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("slots_per_class", C.c_int32), ("steps_per_launch", C.c_int32)]


class _Fields(C.Structure):
    _fields_ = [("eps", C.c_void_p), ("plastic", C.c_void_p), ("labels", C.c_void_p),
                ("on_device", C.c_int32), ("reserved", C.c_int32)]


RECORD_DTYPE = np.dtype([("sig_mean", "f8", 4), ("eps_mean", "f8", 4), ("eta1", "f8"), ("eta2", "f8"),
                         ("eta3", "f8"), ("iterations", "i4"), ("n_plastic", "i4"),
                         ("n_clusters", "i4"), ("status", "i4")])
assert RECORD_DTYPE.itemsize == 104

_lib = None


def lib():
    """The loaded library; raises if it is missing (no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_0802_2488_gb300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i32, dbl = C.c_void_p, C.c_int32, C.c_double
        L.epfft_create.argtypes = [C.POINTER(vp), C.POINTER(_Options)]
        L.epfft_destroy.argtypes = [vp]
        L.epfft_destroy.restype = None
        L.epfft_strerror.argtypes = [C.c_int]
        L.epfft_strerror.restype = C.c_char_p
        L.epfft_supported.argtypes = [i32, i32]
        L.epfft_last_stats.argtypes = [vp, C.POINTER(_Stats)]
        L.epfft_solve.argtypes = [vp, C.POINTER(_Problem), C.POINTER(_Path), vp, C.POINTER(_Fields)]
        L.epfft_solve_dg2.argtypes = [vp, C.POINTER(_Problem), C.POINTER(_Path), vp, C.POINTER(_Fields)]
        L.epfft_average5.argtypes = [vp, i32, i32, vp, vp]
        L.epfft_void_plastic.argtypes = [vp, i32, i32, vp, vp, vp, vp]
        L.epfft_indicators.argtypes = [i32, vp, vp, i32, i32, vp]
        L.epfft_effective_moduli.argtypes = [vp, C.POINTER(_Problem), C.c_double, C.POINTER(C.c_double),
                                             C.POINTER(C.c_double)]
        L.epfft_empirical_curve.argtypes = [i32, vp, vp, i32, C.c_double, i32, C.POINTER(C.c_double), vp]
        L.epfft_eps_eq.argtypes = [vp, i32, i32, vp, vp]
        L.epfft_displacement.argtypes = [vp, i32, i32, vp, vp]
        L.epfft_solve_batch.argtypes = [vp, i32, C.POINTER(_Problem), C.POINTER(_Path), C.POINTER(vp),
                                        C.POINTER(_Fields)]
        L.epfft_mask.argtypes = [i32, dbl, C.c_uint64, vp, vp]
        L.epfft_iterate.argtypes = [vp, C.POINTER(_Problem), C.POINTER(dbl), vp, i32, vp]
        L.epfft_project.argtypes = [vp, i32, i32, dbl, dbl, C.POINTER(dbl), vp, vp]
        L.epfft_label.argtypes = [vp, i32, i32, vp, i32, vp, vp]
        L.epfft_serve_open.argtypes = [vp, C.POINTER(_ServeOptions)]
        L.epfft_serve_close.argtypes = [vp]
        L.epfft_submit.argtypes = [vp, C.POINTER(_Problem), C.POINTER(_Path), i32, C.POINTER(C.c_int64)]
        L.epfft_serve_step.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
        L.epfft_poll.argtypes = [vp, C.c_int64, vp, vp, C.POINTER(dbl)]
        L.epfft_ticket_fields.argtypes = [vp, C.c_int64, i32, vp, vp, vp, vp]
        L.epfft_release.argtypes = [vp, C.c_int64]
        L.epfft_solve_refined.argtypes = [vp, C.POINTER(_Problem), C.POINTER(_Path), dbl, vp, vp, vp]
        L.epfft_solve_refined_batch.argtypes = [vp, i32, vp, vp, dbl, vp, vp, vp]
        L.epfft_autotune.argtypes = [vp, i32, i32, i32, C.POINTER(i32), C.POINTER(C.c_float)]
        L.epfft_set_tiling.argtypes = [vp, i32, i32, i32]
        L.epfft_set_defect_refresh.argtypes = [vp, i32]
        L.epfft_project_static.argtypes = [i32, i32, dbl, dbl, C.POINTER(dbl), vp, vp, vp]
        L.epfft_time_passes.argtypes = [vp, C.POINTER(_Problem), i32, C.POINTER(dbl), i32, C.POINTER(C.c_float),
                                        C.POINTER(C.c_float)]
        L.epfft_fp64_peak.argtypes = [vp, C.POINTER(dbl), C.POINTER(i32), C.POINTER(C.c_float)]
        L.epfft_supported_tiling.argtypes = [i32, i32, i32]
        for s in SYMBOLS:
            if s not in ("epfft_destroy", "epfft_strerror"):
                getattr(L, s).restype = C.c_int
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().epfft_strerror(int(code)).decode()


def _check(rc: int, what: str, allow=(EPFFT_OK,)) -> int:
    if rc not in allow:
        raise EpfftError(rc, what)
    return rc


# --------------------------------------------------------------------------
# Problem description (Sec. 2) and the default material of the workloads
# --------------------------------------------------------------------------

@dataclass
class Problem:
    L: int
    precision: str = "fp64"          # 'fp64' | 'fp32' | 'fp32_defect'
    void_fraction: float = 0.0
    seed: int = 0
    mask: Optional[object] = None    # numpy uint8 (L, L) or torch CUDA uint8 tensor; None: generated
    mu: float = 1.0
    lambda_: float = 1.5
    yield_stress: float = 1.0
    mu0: Optional[float] = None      # reference medium; None: the matrix moduli
    lambda0: Optional[float] = None
    tol_eq: float = 1e-8
    tol_macro: float = 1e-8
    max_iter: int = 10000
    green: str = "eq3"               # 'eq3' | 'cg1' | 'dg1' (Sec. 2)
    eq_test: str = "own"             # 'own' (eta1 for Eq. 3, eta3 for CG1/DG1) | 'fixed_point' (eta3 for all)

    def _c(self) -> tuple[_Problem, object]:
        keep = None
        mptr, mdev = None, 0
        if self.mask is not None:
            if isinstance(self.mask, np.ndarray):
                keep = np.ascontiguousarray(self.mask, dtype=np.uint8)
                assert keep.size == self.L * self.L
                mptr = keep.ctypes.data
            else:  # torch tensor on the device
                keep = self.mask.contiguous()
                assert keep.is_cuda and keep.numel() == self.L * self.L
                mptr, mdev = keep.data_ptr(), 1
        prec = _PREC[self.precision]
        p = _Problem(self.L, prec, float(self.void_fraction), int(self.seed) & (2**64 - 1), mptr, mdev,
                     _GREEN[self.green], self.mu, self.lambda_, self.yield_stress,
                     self.mu if self.mu0 is None else self.mu0,
                     self.lambda_ if self.lambda0 is None else self.lambda0,
                     self.tol_eq, self.tol_macro, int(self.max_iter), _EQ_TEST[self.eq_test])
        return p, keep

    @property
    def real_dtype(self):
        return np.float32 if self.precision == "fp32" else np.float64


def _path(E) -> tuple[_Path, np.ndarray]:
    a = np.ascontiguousarray(E, dtype=np.float64).reshape(-1, 4)
    return _Path(a.shape[0], 0, a.ctypes.data), a


# --------------------------------------------------------------------------
# Context (epfft_create / epfft_destroy)
# --------------------------------------------------------------------------

class Context:
    """epfft_ctx on one CUDA device, allocating through torch's caching
    allocator; it works on `stream` (a cudaStream_t as int, e.g.
    torch.cuda.Stream().cuda_stream) or on a stream of its own."""

    def __init__(self, device: int = 0, torch_allocator: bool = True, stream: Optional[int] = None):
        import torch
        self.device = device
        self._torch = torch
        torch.cuda.init()
        self.handle = C.c_void_p()
        if torch_allocator:
            def _alloc(nbytes, stream, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0)
                except Exception:
                    return None

            def _free(ptr, nbytes, stream, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._cbs = (AllocFn(_alloc), FreeFn(_free))
            opts = _Options(device, 0, stream, self._cbs[0], self._cbs[1], None)
        else:
            self._cbs = None
            opts = _Options(device, 0, stream, AllocFn(), FreeFn(), None)
        _check(lib().epfft_create(C.byref(self.handle), C.byref(opts)), "epfft_create")

    def close(self):
        if self.handle:
            lib().epfft_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def epfft_create(device: int = 0) -> Context:
    return Context(device)


def epfft_destroy(ctx: Context) -> None:
    ctx.close()


def epfft_last_stats(ctx: Context) -> dict:
    """Device-loop steps, kernel launches and iterations of the last solve-type call."""
    st = _Stats()
    _check(lib().epfft_last_stats(ctx.handle, C.byref(st)), "epfft_last_stats")
    return {"loop_steps": st.loop_steps, "kernel_launches": st.kernel_launches, "iterations": st.iterations}


def epfft_strerror(code: int) -> str:
    return strerror(code)


def epfft_supported(L: int, precision: str) -> bool:
    return bool(lib().epfft_supported(L, _PREC[precision]))


@dataclass
class Fields:
    eps: Optional[np.ndarray] = None       # (L, L, 4) final local strain
    plastic: Optional[np.ndarray] = None   # (n_inc, L, L) uint8
    labels: Optional[np.ndarray] = None    # (n_inc, L, L) int32


def _c_fields(f: Fields):
    return _Fields(f.eps.ctypes.data, f.plastic.ctypes.data, f.labels.ctypes.data, 0, 0)


def _host_fields(prob: Problem, n_inc: int):
    L = prob.L
    f = Fields(np.empty((L, L, 4), dtype=prob.real_dtype), np.empty((n_inc, L, L), np.uint8),
               np.empty((n_inc, L, L), np.int32))
    return f, _c_fields(f)


def pinned_fields(problem: Problem, n_inc: int) -> Fields:
    """Host output buffers of one solve in page-locked memory (torch's
    pinned allocator), for reuse across calls through `out=`: copies into
    them run at the link's rate instead of through a staging buffer."""
    import torch
    L = problem.L
    tdt = torch.float32 if problem.precision == "fp32" else torch.float64

    def arr(shape, dt):
        return torch.empty(shape, dtype=dt, pin_memory=True).numpy()
    return Fields(arr((L, L, 4), tdt), arr((n_inc, L, L), torch.uint8), arr((n_inc, L, L), torch.int32))


def _check_out(f: Fields, prob: Problem, n_inc: int):
    L = prob.L
    assert f.eps.shape == (L, L, 4) and f.eps.dtype == prob.real_dtype and f.eps.flags["C_CONTIGUOUS"]
    assert f.plastic.shape == (n_inc, L, L) and f.plastic.dtype == np.uint8 and f.plastic.flags["C_CONTIGUOUS"]
    assert f.labels.shape == (n_inc, L, L) and f.labels.dtype == np.int32 and f.labels.flags["C_CONTIGUOUS"]


def epfft_solve(ctx: Context, problem: Problem, path, fields: bool = False):
    """Blocking solve along `path` ((n_inc, 4) mean strains).  Returns
    (rc, records[, Fields]); rc is EPFFT_OK or EPFFT_NOT_CONVERGED."""
    p, keep = problem._c()
    cp, parr = _path(path)
    rec = np.zeros(cp.n_inc, dtype=RECORD_DTYPE)
    f, cf = _host_fields(problem, cp.n_inc) if fields else (None, None)
    rc = lib().epfft_solve(ctx.handle, C.byref(p), C.byref(cp), rec.ctypes.data,
                           C.byref(cf) if cf is not None else None)
    _check(rc, "epfft_solve", (EPFFT_OK, EPFFT_NOT_CONVERGED))
    return (rc, rec, f) if fields else (rc, rec)


def epfft_solve_refined(ctx: Context, problem: Problem, path, tol_switch: float = 0.0, fields: bool = False):
    """Mixed-precision solve: per increment FP32 iterations to
    max(tol_switch, tolerance) (tol_switch = 0: until they stall at the FP32
    floor), then FP64 iterations to the tolerances (problem.precision must be
    'fp64').  Returns (rc, records of the FP64
    stages, records of the FP32 stages[, Fields])."""
    p, keep = problem._c()
    cp, parr = _path(path)
    rec = np.zeros(cp.n_inc, dtype=RECORD_DTYPE)
    rec32 = np.zeros(cp.n_inc, dtype=RECORD_DTYPE)
    f, cf = _host_fields(problem, cp.n_inc) if fields else (None, None)
    rc = lib().epfft_solve_refined(ctx.handle, C.byref(p), C.byref(cp), float(tol_switch), rec.ctypes.data,
                                   rec32.ctypes.data, C.byref(cf) if cf is not None else None)
    _check(rc, "epfft_solve_refined", (EPFFT_OK, EPFFT_NOT_CONVERGED))
    return (rc, rec, rec32, f) if fields else (rc, rec, rec32)


def epfft_solve_refined_batch(ctx: Context, problems: Sequence[Problem], paths: Sequence, tol_switch: float = 0.0):
    """The mixed-precision solve of problems sharing L and the increment
    count, advanced together.  Returns (rc, [FP64-stage records],
    [FP32-stage records])."""
    n = len(problems)
    cps, keeps = zip(*(p._c() for p in problems))
    arr = (_Problem * n)(*cps)
    pth = [_path(P) for P in paths]
    carr = (_Path * n)(*(x[0] for x in pth))
    recs = [np.zeros(x[0].n_inc, dtype=RECORD_DTYPE) for x in pth]
    recs32 = [np.zeros(x[0].n_inc, dtype=RECORD_DTYPE) for x in pth]
    rptr = (C.c_void_p * n)(*(r.ctypes.data for r in recs))
    rptr32 = (C.c_void_p * n)(*(r.ctypes.data for r in recs32))
    rc = lib().epfft_solve_refined_batch(ctx.handle, n, C.cast(arr, C.c_void_p), C.cast(carr, C.c_void_p),
                                         float(tol_switch), C.cast(rptr, C.c_void_p), C.cast(rptr32, C.c_void_p),
                                         None)
    _check(rc, "epfft_solve_refined_batch", (EPFFT_OK, EPFFT_NOT_CONVERGED))
    return rc, recs, recs32


def epfft_solve_dg2(ctx: Context, problem: Problem, path, fields: bool = False):
    """DG2 (Sec. 2): the average of four complete solves with the Eq. 3
    operator at mirrored momenta.  Returns (rc, records[, Fields]) with
    Fields.eps the averaged final strain and Fields.plastic / labels (L, L)
    arrays of that field's plastic pixels and their clusters."""
    p, keep = problem._c()
    cp, parr = _path(path)
    rec = np.zeros(cp.n_inc, dtype=RECORD_DTYPE)
    f = cf = None
    if fields:
        L = problem.L
        f = Fields(np.empty((L, L, 4), dtype=problem.real_dtype), np.empty((L, L), np.uint8),
                   np.empty((L, L), np.int32))
        cf = _Fields(f.eps.ctypes.data, f.plastic.ctypes.data, f.labels.ctypes.data, 0, 0)
    rc = lib().epfft_solve_dg2(ctx.handle, C.byref(p), C.byref(cp), rec.ctypes.data,
                               C.byref(cf) if cf is not None else None)
    _check(rc, "epfft_solve_dg2", (EPFFT_OK, EPFFT_NOT_CONVERGED))
    return (rc, rec, f) if fields else (rc, rec)


def epfft_void_plastic(ctx: Context, mask, plastic, labels: bool = False):
    """Sec. 3 void-plastic clusters.  mask: (L, L) uint8, plastic: (L, L) or
    (n, L, L) uint8, numpy or CUDA tensors.  Returns stats (n, 6) int32
    [, labels (n, L, L) int32 CUDA tensor]."""
    import torch
    m = torch.as_tensor(mask, dtype=torch.uint8).to("cuda").contiguous()
    p = torch.as_tensor(plastic, dtype=torch.uint8).to("cuda").contiguous()
    L = m.shape[-1]
    n = p.numel() // (L * L)
    lab = torch.empty((n, L, L), dtype=torch.int32, device="cuda") if labels else None
    st = np.zeros((n, 6), dtype=np.int32)
    torch.cuda.current_stream().synchronize()
    _check(lib().epfft_void_plastic(ctx.handle, L, n, m.data_ptr(), p.data_ptr(),
                                    lab.data_ptr() if labels else None, st.ctypes.data), "epfft_void_plastic")
    return (st, lab) if labels else st


def epfft_indicators(records, stats, L: int, load: str) -> np.ndarray:
    """Sec. 3 indicators per increment, (n_inc, 8): eps0, sigma0, f_p, v_max,
    i, n, r, -d2 sigma0 / d eps0^2 (computed by the library)."""
    rec = np.ascontiguousarray(records, dtype=RECORD_DTYPE)
    st = np.ascontiguousarray(stats, dtype=np.int32)
    out = np.zeros((len(rec), 8))
    _check(lib().epfft_indicators(len(rec), rec.ctypes.data, st.ctypes.data, L,
                                  {"equibiaxial": 0, "shear": 1}[load], out.ctypes.data), "epfft_indicators")
    return out


def epfft_effective_moduli(ctx: Context, problem: Problem, strain: float = 1e-3):
    """(K~, mu~) of the lattice with the elastic matrix (Eqs. 5-6)."""
    p, keep = problem._c()
    K, mu = C.c_double(), C.c_double()
    rc = lib().epfft_effective_moduli(ctx.handle, C.byref(p), float(strain), C.byref(K), C.byref(mu))
    _check(rc, "epfft_effective_moduli", (EPFFT_OK, EPFFT_NOT_CONVERGED))
    return K.value, mu.value


def epfft_empirical_curve(ind, stats, L: int, modulus: float, load: str):
    """Eqs. 5-6: (alpha, fitted sigma0 per increment)."""
    a = np.ascontiguousarray(ind, dtype=np.float64)
    st = np.ascontiguousarray(stats, dtype=np.int32)
    fit = np.zeros(len(a))
    alpha = C.c_double()
    _check(lib().epfft_empirical_curve(len(a), a.ctypes.data, st.ctypes.data, L, float(modulus),
                                       {"equibiaxial": 0, "shear": 1}[load], C.byref(alpha), fit.ctypes.data),
           "epfft_empirical_curve")
    return alpha.value, fit


def epfft_eps_eq(ctx: Context, L: int, precision: str, eps):
    """Equivalent strain field (Fig. 1) of a CUDA strain tensor (L, L, 4)."""
    import torch
    assert eps.is_cuda and eps.is_contiguous() and eps.numel() == 4 * L * L
    out = torch.empty((L, L), dtype=eps.dtype, device=eps.device)
    _check(lib().epfft_eps_eq(ctx.handle, L, _PREC[precision],
                              eps.data_ptr(), out.data_ptr()), "epfft_eps_eq")
    return out


def epfft_displacement(ctx: Context, L: int, precision: str, eps):
    """Displacement field (Sec. 2) of a CUDA strain tensor (L, L, 4): a CUDA
    tensor (L, L, 2) of (u1, u2) with zero mean."""
    import torch
    assert eps.is_cuda and eps.is_contiguous() and eps.numel() == 4 * L * L
    assert eps.dtype == (torch.float64 if precision == "fp64" else torch.float32)
    u = torch.empty((L, L, 2), dtype=eps.dtype, device=eps.device)
    _check(lib().epfft_displacement(ctx.handle, L, _PREC[precision],
                                    eps.data_ptr(), u.data_ptr()), "epfft_displacement")
    return u


def epfft_average5(ctx: Context, L: int, precision: str, eps_in, eps_out):
    """CG2 post-processing (Sec. 2) of a device strain field: eps_out = mean of
    each pixel and its four neighbours.  eps_in / eps_out: CUDA tensors of
    L*L*4 reals."""
    assert eps_in.is_cuda and eps_out.is_cuda and eps_in.numel() == eps_out.numel() == L * L * 4
    _check(lib().epfft_average5(ctx.handle, L, _PREC[precision],
                                eps_in.data_ptr(), eps_out.data_ptr()), "epfft_average5")


def epfft_solve_batch(ctx: Context, problems: Sequence[Problem], paths: Sequence, fields: bool = False,
                      out: Optional[Sequence[Fields]] = None):
    """Blocking solve of problems advanced together in one device loop (one
    graph launch; problems of differing L or precision run on parallel
    branches of its body).  Returns (rc, [records][, [Fields]]).  With fields,
    `out` may give the host buffers to fill (one Fields per problem, e.g.
    from pinned_fields); otherwise new arrays are allocated."""
    n = len(problems)
    cps, keeps = zip(*(p._c() for p in problems))
    arr = (_Problem * n)(*cps)
    pth = [_path(P) for P in paths]
    carr = (_Path * n)(*(x[0] for x in pth))
    recs = [np.zeros(x[0].n_inc, dtype=RECORD_DTYPE) for x in pth]
    rptr = (C.c_void_p * n)(*(r.ctypes.data for r in recs))
    if fields:
        if out is not None:
            assert len(out) == n
            for i in range(n):
                _check_out(out[i], problems[i], pth[i][0].n_inc)
            fl = [(out[i], _c_fields(out[i])) for i in range(n)]
        else:
            fl = [_host_fields(problems[i], pth[i][0].n_inc) for i in range(n)]
        farr = (_Fields * n)(*(x[1] for x in fl))
    rc = lib().epfft_solve_batch(ctx.handle, n, arr, carr, rptr, farr if fields else None)
    _check(rc, "epfft_solve_batch", (EPFFT_OK, EPFFT_NOT_CONVERGED))
    return (rc, recs, [x[0] for x in fl]) if fields else (rc, recs)


def epfft_mask(L: int, void_fraction: float, seed: int, device: int = 0):
    """Void mask of Sec. 2 as a torch uint8 (L, L) CUDA tensor."""
    import torch
    m = torch.empty((L, L), dtype=torch.uint8, device=f"cuda:{device}")
    s = torch.cuda.current_stream(device)
    _check(lib().epfft_mask(L, float(void_fraction), int(seed) & (2**64 - 1), m.data_ptr(), s.cuda_stream),
           "epfft_mask")
    return m


def epfft_iterate(ctx: Context, problem: Problem, E, eps, n_iter: int):
    """n_iter AL iterations from the CUDA tensor eps ((L, L, 4), the
    problem's real dtype), in place.  Returns the record of the last iterate."""
    import torch
    p, keep = problem._c()
    assert eps.is_cuda and eps.is_contiguous() and eps.numel() == 4 * problem.L ** 2
    assert eps.dtype == (torch.float32 if problem.precision == "fp32" else torch.float64)
    Ea = (C.c_double * 4)(*[float(x) for x in E])
    rec = np.zeros(1, dtype=RECORD_DTYPE)
    torch.cuda.current_stream(ctx.device).synchronize()
    _check(lib().epfft_iterate(ctx.handle, C.byref(p), Ea, eps.data_ptr(), int(n_iter), rec.ctypes.data),
           "epfft_iterate")
    return rec[0]


def epfft_project(ctx: Context, L: int, precision: str, lambda0: float, mu0: float, E, p):
    """e = E + IDFT(G DFT(p)) (Eqs. 2-3) for a CUDA tensor p (3, L, L)."""
    import torch
    assert p.is_cuda and p.is_contiguous() and tuple(p.shape) == (3, L, L)
    e = torch.empty_like(p)
    Ea = (C.c_double * 4)(*[float(x) for x in E])
    torch.cuda.current_stream(ctx.device).synchronize()
    _check(lib().epfft_project(ctx.handle, L, _PREC[precision],
                               float(lambda0), float(mu0), Ea, p.data_ptr(), e.data_ptr()), "epfft_project")
    return e


def epfft_label(ctx: Context, flags, periodic: bool = True):
    """Clusters of flagged pixels of a CUDA uint8 tensor (n, L, L).
    Returns (labels int32 tensor, counts numpy)."""
    import torch
    assert flags.is_cuda and flags.dtype == torch.uint8 and flags.is_contiguous()
    n, L, L2 = flags.shape
    assert L == L2
    lab = torch.empty((n, L, L), dtype=torch.int32, device=flags.device)
    counts = np.zeros(n, dtype=np.int32)
    torch.cuda.current_stream(ctx.device).synchronize()
    _check(lib().epfft_label(ctx.handle, L, n, flags.data_ptr(), 1 if periodic else 0, lab.data_ptr(),
                             counts.ctypes.data), "epfft_label")
    return lab, counts


def epfft_time_passes(ctx: Context, problem: Problem, E, n_iter: int, n_batch: int = 1):
    """(column-pass ms, row-pass ms): mean CUDA-event durations over n_iter
    launches of each for a batch of n_batch copies, from the state eps = E."""
    p, keep = problem._c()
    Ea = (C.c_double * 4)(*[float(x) for x in E])
    a, b = C.c_float(), C.c_float()
    _check(lib().epfft_time_passes(ctx.handle, C.byref(p), int(n_batch), Ea, int(n_iter), C.byref(a),
                                   C.byref(b)), "epfft_time_passes")
    return a.value, b.value


def epfft_fp64_peak(ctx: Context) -> dict:
    """Measured FP64 FMA throughput of the context's device (TFLOP/s), its SM
    count and the best launch time (ms)."""
    t, n, ms = C.c_double(), C.c_int32(), C.c_float()
    _check(lib().epfft_fp64_peak(ctx.handle, C.byref(t), C.byref(n), C.byref(ms)), "epfft_fp64_peak")
    return {"tflops": t.value, "n_sm": n.value, "ms": ms.value}


def epfft_project_static(L: int, precision: str, lambda0: float, mu0: float, E, p, stream=None, out=None,
                         wait: bool = True):
    """epfft_project without any device allocation by the library: its working
    memory is a static device array (lattice sides up to 256).  The output
    tensor is `out` if given, else allocated here by torch before the call;
    the library queues its work on `stream` (default: torch's current stream)
    and this wrapper waits for it unless wait=False."""
    import torch
    assert p.is_cuda and p.is_contiguous() and tuple(p.shape) == (3, L, L)
    e = torch.empty_like(p) if out is None else out
    assert e.is_cuda and e.is_contiguous() and e.shape == p.shape and e.dtype == p.dtype
    Ea = (C.c_double * 4)(*[float(x) for x in E])
    s = torch.cuda.current_stream(p.device) if stream is None else stream
    _check(lib().epfft_project_static(L, _PREC[precision], float(lambda0),
                                      float(mu0), Ea, p.data_ptr(), e.data_ptr(), s.cuda_stream),
           "epfft_project_static")
    if wait:
        s.synchronize()
    return e


# --------------------------------------------------------------------------
# Serving (continuous batching)
# --------------------------------------------------------------------------

def epfft_serve_open(ctx: Context, hbm_budget_bytes: int, slots_per_class: int = 16, steps_per_launch: int = 64):
    _check(lib().epfft_serve_open(ctx.handle, C.byref(_ServeOptions(int(hbm_budget_bytes), int(slots_per_class),
                                                                     int(steps_per_launch)))), "epfft_serve_open")


def epfft_serve_close(ctx: Context):
    _check(lib().epfft_serve_close(ctx.handle), "epfft_serve_close")


def epfft_submit(ctx: Context, problem: Problem, path, want_eps: bool = False, want_sig: bool = False,
                 want_plastic: bool = False, want_labels: bool = False) -> int:
    """Queues one solve; the want_* flags choose the fields kept for the
    caller (the final strain through epfft_poll; the final stress and the
    per-increment plastic flags and cluster labels through
    epfft_ticket_fields, until epfft_release)."""
    p, keep = problem._c()
    cp, parr = _path(path)
    want = ((EPFFT_WANT_EPS if want_eps else 0) | (EPFFT_WANT_SIG if want_sig else 0) |
            (EPFFT_WANT_PLASTIC if want_plastic else 0) | (EPFFT_WANT_LABELS if want_labels else 0))
    t = C.c_int64()
    _check(lib().epfft_submit(ctx.handle, C.byref(p), C.byref(cp), want, C.byref(t)), "epfft_submit")
    return t.value


def epfft_serve_step(ctx: Context) -> tuple[int, int]:
    """One admission / device / harvest round; returns (running, queued)."""
    r, q = C.c_int32(), C.c_int32()
    _check(lib().epfft_serve_step(ctx.handle, C.byref(r), C.byref(q)), "epfft_serve_step")
    return r.value, q.value


def epfft_poll(ctx: Context, ticket: int, problem: Problem, n_inc: int, want_eps: bool = False):
    """None while pending; else (rc, records, eps or None, latency seconds)."""
    rec = np.zeros(n_inc, dtype=RECORD_DTYPE)
    eps = np.empty((problem.L, problem.L, 4), dtype=problem.real_dtype) if want_eps else None
    lat = C.c_double()
    rc = lib().epfft_poll(ctx.handle, int(ticket), rec.ctypes.data, eps.ctypes.data if eps is not None else None,
                          C.byref(lat))
    if rc == EPFFT_PENDING:
        return None
    _check(rc, "epfft_poll", (EPFFT_OK, EPFFT_NOT_CONVERGED))
    return rc, rec, eps, lat.value


def epfft_ticket_fields(ctx: Context, ticket: int, problem: Problem, inc: int, eps: bool = False,
                        sig: bool = False, plastic: bool = False, labels: bool = False) -> Optional[dict]:
    """Fields of a finished served solve at increment inc (eps and sig: the
    final accepted state, inc = n_inc - 1 only), as numpy arrays keyed
    'eps', 'sig', 'plastic', 'labels'; None while it is pending."""
    L = problem.L
    out = {}
    if eps:
        out["eps"] = np.empty((L, L, 4), dtype=problem.real_dtype)
    if sig:
        out["sig"] = np.empty((L, L, 4), dtype=problem.real_dtype)
    if plastic:
        out["plastic"] = np.empty((L, L), dtype=np.uint8)
    if labels:
        out["labels"] = np.empty((L, L), dtype=np.int32)
    ptr = lambda k: out[k].ctypes.data if k in out else None
    rc = lib().epfft_ticket_fields(ctx.handle, int(ticket), int(inc), ptr("eps"), ptr("sig"), ptr("plastic"),
                                   ptr("labels"))
    if rc == EPFFT_PENDING:
        return None
    _check(rc, "epfft_ticket_fields")
    return out


def epfft_release(ctx: Context, ticket: int) -> bool:
    """Releases a finished ticket and its fields; False while it is pending."""
    rc = lib().epfft_release(ctx.handle, int(ticket))
    if rc == EPFFT_PENDING:
        return False
    _check(rc, "epfft_release")
    return True


# --------------------------------------------------------------------------
# Tiling
# --------------------------------------------------------------------------

def epfft_autotune(ctx: Context, L: int, precision: str, n_batch: int = 1):
    """Times the compiled tilings of (L, precision) on a batch of n_batch
    solves and keeps the faster for the context (for batches of that size
    class).  Returns (chosen tiling, [ms per iteration of each])."""
    ch = C.c_int32()
    ms = (C.c_float * N_TILINGS)()
    _check(lib().epfft_autotune(ctx.handle, L, _PREC[precision], int(n_batch),
                                C.byref(ch), ms), "epfft_autotune")
    return ch.value, list(ms)


def epfft_supported_tiling(L: int, precision: str, variant: int) -> bool:
    return bool(lib().epfft_supported_tiling(L, _PREC[precision], int(variant)))


def epfft_set_tiling(ctx: Context, L: int, precision: str, variant: int):
    _check(lib().epfft_set_tiling(ctx.handle, L, _PREC[precision], int(variant)),
           "epfft_set_tiling")


def epfft_set_defect_refresh(ctx: Context, steps: int):
    """Loop steps between refreshes of the FP64 reference of the defect
    form ('fp32_defect'); 1 makes every iteration the FP64 one."""
    _check(lib().epfft_set_defect_refresh(ctx.handle, int(steps)), "epfft_set_defect_refresh")
