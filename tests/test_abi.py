"""CPU checks of the C ABI library: it builds, loads without a GPU and exports
every function include/s2let_gpu.h declares; host-only entry points work."""
import os
import re

import pytest

from paper_1211_1680_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "s2let_gpu.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(s2let_\w+)\s*\(", txt)))


def test_library_builds_and_loads():
    build.build()
    assert os.path.exists(build.LIB)
    assert _lib.lib() is not None


def test_exports_every_declared_symbol():
    names = _declared()
    assert len(names) >= 10
    L = _lib.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(_lib.SIGNATURES)


def test_host_entry_points():
    L = _lib.lib()
    assert L.s2let_jmax(2048, 2) == 11
    assert L.s2let_jmax(128, 3) == 5
    assert L.s2let_jmax(3, 2) == 1
    assert L.s2let_jmax(1, 2) == _lib.S2LET_ERR_ARG
    assert L.s2let_strerror(0) == b"ok"


def test_plan_argument_errors_need_no_gpu():
    import ctypes
    L = _lib.lib()
    h = ctypes.c_void_p()
    # J_min must be < J (Sect. 2.2); these are rejected before any CUDA call
    assert L.s2let_plan_create(ctypes.byref(h), 32, 2, 5, 0, 1) == _lib.S2LET_ERR_ARG
    assert L.s2let_plan_create(ctypes.byref(h), 2, 2, 0, 0, 1) == _lib.S2LET_ERR_ARG
    assert L.s2let_plan_create(ctypes.byref(h), 32, 1, 0, 0, 1) == _lib.S2LET_ERR_ARG
    assert L.s2let_plan_create(ctypes.byref(h), 32, 2, 0, 0x2000, 1) == _lib.S2LET_ERR_ARG
    # the Legendre-table switch belongs to TF32X3 plans only
    for prec in (_lib.S2LET_PREC_FP64, _lib.S2LET_PREC_FP32):
        assert L.s2let_plan_create(ctypes.byref(h), 32, 2, 0, prec | _lib.S2LET_LEG_RECURRENCE,
                                   1) == _lib.S2LET_ERR_ARG
    assert L.s2let_plan_create(ctypes.byref(h), 4097, 2, 0, _lib.S2LET_PREC_TF32X3, 1) == _lib.S2LET_ERR_ARG
    # FP64 plans stop at L = 2048 (their shared-memory FFTs), FP32 / TF32X3 plans at 4096
    assert L.s2let_plan_create(ctypes.byref(h), 4096, 2, 0, 0, 1) == _lib.S2LET_ERR_UNSUPPORTED
    assert L.s2let_plan_create(ctypes.byref(h), 2049, 2, 0, _lib.S2LET_PREC_FP32 | _lib.S2LET_QUAD_FFT64,
                               1) == _lib.S2LET_ERR_UNSUPPORTED
    assert L.s2let_plan_create(ctypes.byref(h), 32, 2, 0, 0, 0) == _lib.S2LET_ERR_ARG
    assert not h.value


def test_flag_constants_match_header():
    """Every S2LET_* constant the header defines has the same value in the binding."""
    txt = open(os.path.join(ROOT, "include", "s2let_gpu.h")).read()
    defs = {k: int(v, 0) for k, v in re.findall(r"#define\s+(S2LET_\w+)\s+\(?(-?(?:0x)?[0-9a-fA-F]+)\)?", txt)}
    assert "S2LET_KERNEL_BSPLINE" in defs and "S2LET_PREC_TF32X3" in defs
    for k, v in defs.items():
        if hasattr(_lib, k):
            assert getattr(_lib, k) == v, k
    for k in ("S2LET_COMPLEX", "S2LET_MULTIRES", "S2LET_PREC_FP32", "S2LET_PREC_TF32X3", "S2LET_QUAD_FFT64",
              "S2LET_TC_SPLIT3", "S2LET_KERNEL_BSPLINE", "S2LET_LEG_RECURRENCE", "S2LET_ERR_ARG"):
        assert getattr(_lib, k) == defs[k], k


def test_binding_rejects_unknown_kernel_family_without_gpu():
    from paper_1211_1680_gb300.s2let import BatchPlan, Plan
    with pytest.raises(ValueError):
        Plan(32, 2, 0, kernel="needlet")
    with pytest.raises(ValueError):
        BatchPlan([32], [2], 0, kernel="spline")


def test_allocator_hook_arguments_need_no_gpu():
    L = _lib.lib()
    a = _lib.ALLOC_FN(lambda n, c: None)
    assert L.s2let_set_allocator(a, _lib.FREE_FN(), None) == _lib.S2LET_ERR_ARG
    assert L.s2let_set_allocator(_lib.ALLOC_FN(), _lib.FREE_FN(), None) == _lib.S2LET_OK
