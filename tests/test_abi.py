"""The C ABI library loads and exports every entry point include/epfft.h
declares; its host-only calls work without a GPU (no compute is launched)."""
import os
import re

import pytest

from paper_0802_2488_gb300 import binding as B
from paper_0802_2488_gb300 import build as build_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "epfft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(epfft_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return B.lib()


def test_every_declared_entry_point_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(B.SYMBOLS) == names


def test_binding_keeps_the_c_names():
    for n in declared_symbols():
        assert callable(getattr(B, n)), n


def test_host_only_calls(lib):
    assert B.strerror(B.EPFFT_OK) == "ok"
    assert "argument" in B.strerror(B.EPFFT_ERR_ARG)
    assert B.epfft_supported(256, "fp64") and B.epfft_supported(4096, "fp32") and B.epfft_supported(4096, "fp64")
    assert not B.epfft_supported(8192, "fp64") and not B.epfft_supported(8192, "fp32")
    assert lib.epfft_supported(100, 1) == 0 and lib.epfft_supported(2, 1) == 0
    # the defect-correction form: where both the FP32 passes and the FP64
    # refresh are built, tilings 0 and 1 only
    assert B.epfft_supported(4096, "fp32_defect") and not B.epfft_supported(8192, "fp32_defect")
    assert B.epfft_supported_tiling(512, "fp32_defect", 1) and not B.epfft_supported_tiling(512, "fp32_defect", 2)
    assert lib.epfft_supported(256, 3) == 0
    # the on-chip schedule: FP32, sides 16 .. 64
    assert [B.epfft_supported_tiling(L, "fp32", 3) for L in (8, 16, 32, 64, 128)] == [False, True, True, True, False]
    assert not B.epfft_supported_tiling(64, "fp64", 3) and not B.epfft_supported_tiling(64, "fp32_defect", 3)
    assert lib.epfft_set_defect_refresh(None, 8) == B.EPFFT_ERR_ARG


def test_no_cpu_fallback_without_device(lib):
    import ctypes as C
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    rc = lib.epfft_create(C.byref(h), None)
    assert rc == B.EPFFT_ERR_CUDA and not h.value


def test_argument_checks_of_analysis_entry_points(lib):
    """Host-side argument checks of the Sec. 3 / Eqs. 5-6 entry points reject
    bad input before any device work."""
    import ctypes as C
    import numpy as np
    out = np.zeros(8)
    rec = np.zeros(2, dtype=B.RECORD_DTYPE)
    st = np.zeros((2, 6), np.int32)
    ok = lib.epfft_indicators(2, rec.ctypes.data, st.ctypes.data, 8, 0, np.zeros(16).ctypes.data)
    assert ok == B.EPFFT_OK
    assert lib.epfft_indicators(0, rec.ctypes.data, st.ctypes.data, 8, 0, out.ctypes.data) == B.EPFFT_ERR_ARG
    assert lib.epfft_indicators(2, rec.ctypes.data, st.ctypes.data, 8, 2, out.ctypes.data) == B.EPFFT_ERR_ARG
    assert lib.epfft_indicators(2, None, st.ctypes.data, 8, 0, out.ctypes.data) == B.EPFFT_ERR_ARG
    a = C.c_double()
    ind = np.zeros((2, 8))
    assert lib.epfft_empirical_curve(2, ind.ctypes.data, st.ctypes.data, 8, C.c_double(1.0), 3, C.byref(a),
                                     np.zeros(2).ctypes.data) == B.EPFFT_ERR_ARG
    assert lib.epfft_empirical_curve(0, ind.ctypes.data, st.ctypes.data, 8, C.c_double(1.0), 0, C.byref(a),
                                     np.zeros(2).ctypes.data) == B.EPFFT_ERR_ARG
    # entry points that need a context refuse a null one
    assert lib.epfft_void_plastic(None, 8, 1, None, None, None, None) == B.EPFFT_ERR_ARG
    assert lib.epfft_solve_dg2(None, None, None, None, None) == B.EPFFT_ERR_ARG
    assert lib.epfft_average5(None, 8, 0, None, None) == B.EPFFT_ERR_ARG
    assert lib.epfft_eps_eq(None, 8, 0, None, None) == B.EPFFT_ERR_ARG
    assert lib.epfft_displacement(None, 8, 0, None, None) == B.EPFFT_ERR_ARG
    assert lib.epfft_ticket_fields(None, 0, 0, None, None, None, None) == B.EPFFT_ERR_ARG
    assert lib.epfft_release(None, 0) == B.EPFFT_ERR_ARG
    assert lib.epfft_solve_refined(None, None, None, C.c_double(1e-6), None, None, None) == B.EPFFT_ERR_ARG
    assert lib.epfft_solve_refined_batch(None, 1, None, None, C.c_double(0.0), None, None, None) == B.EPFFT_ERR_ARG
    assert lib.epfft_effective_moduli(None, None, C.c_double(1e-3), None, None) == B.EPFFT_ERR_ARG


def test_binding_constants_match_the_header():
    """Every integer #define of include/epfft.h that the binding names has
    the header's value (status codes, precisions, operators, tests)."""
    src = open(os.path.join(ROOT, "include", "epfft.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(EPFFT_\w+)\s+\(?(-?\d+)\)?", src)}
    assert "EPFFT_EQ_FIXED_POINT" in defs and "EPFFT_GREEN_DG1" in defs and "EPFFT_FP32_DEFECT" in defs
    named = [k for k in defs if hasattr(B, k)]
    assert len(named) >= 10
    for k in named:
        assert getattr(B, k) == defs[k], k
