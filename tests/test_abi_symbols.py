"""The C-ABI library loads on a machine without a GPU and exports every
function that include/mmot.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mmot.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mmot_[a-z0-9_]+)\s*\(", src)))


def test_header_lists_the_boundary():
    names = _declared()
    for required in ("mmot_plan_create", "mmot_marginal", "mmot_sinkhorn_step", "mmot_solve",
                     "mmot_destroy", "mmot_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2405_19246_gb300 import _build, _native
    path = _build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_native.EXPORTED) == set(_declared())


def test_no_cpu_fallback_when_library_missing(monkeypatch):
    from paper_2405_19246_gb300 import _native
    monkeypatch.setattr(_native, "_lib", None)
    monkeypatch.setattr(_native, "LIB_PATH", os.path.join(ROOT, "does_not_exist.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _native.lib()


def test_last_error_without_gpu():
    from paper_2405_19246_gb300 import _build, _native
    _build.build()
    L = _native.lib()
    # invalid arguments are rejected before any CUDA call
    h = ctypes.c_void_p()
    st = L.mmot_plan_create(1, None, None, None, 0.1, 1, 0, None, ctypes.byref(h))
    assert st == 1
    assert b"l = 1" in L.mmot_last_error()
    L.mmot_destroy(None)


def test_batch_rejects_bad_arguments_without_gpu():
    from paper_2405_19246_gb300 import _build, _native
    _build.build()
    L = _native.lib()
    h = ctypes.c_void_p()
    assert L.mmot_batch_create(0, None, None, None, None, None, 1, 0, None, ctypes.byref(h)) == 1
    ls = (ctypes.c_int * 2)(3, 9)
    N = (ctypes.c_int64 * 12)(*([4] * 12))
    X = (ctypes.c_void_p * 12)()
    eps = (ctypes.c_double * 2)(0.1, 0.1)
    st = L.mmot_batch_create(2, ls, N, X, X, eps, 1, 0, None, ctypes.byref(h))
    assert st == 1
    assert b"instance 1: l = 9" in L.mmot_last_error()
    assert L.mmot_batch_create(2, ls, N, X, X, eps, 1, -1, None, ctypes.byref(h)) == 1
    L.mmot_batch_destroy(None)


def test_memory_limit_arguments_without_gpu():
    from paper_2405_19246_gb300 import _build, _native
    _build.build()
    L = _native.lib()
    assert L.mmot_set_memory_limit(-1) == 1
    assert b"memory limit" in L.mmot_last_error()
    assert L.mmot_set_memory_limit(0) == 0
    used = ctypes.c_int64(-1)
    assert L.mmot_memory_in_use(ctypes.byref(used)) == 0
    assert used.value == 0   # no plan exists in this process
    assert L.mmot_memory_in_use(None) == 1
