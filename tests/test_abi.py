"""The C-ABI library builds, loads and exports every symbol include/brahmap.h
declares (no GPU needed; no compute calls)."""
import os

import pytest

import paper_2501_16122_gb300 as pkg


@pytest.fixture(scope="module")
def L():
    pkg.build()
    from paper_2501_16122_gb300 import _lib
    return _lib


def test_every_declared_symbol_is_exported(L):
    names = L.header_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L.lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_function(L):
    for n in L.header_functions():
        assert hasattr(L, n) or n in ("bm_status_string",), n


def test_status_strings_and_version(L):
    assert L.status_string(L.BM_OK) == "ok"
    assert L.status_string(L.BM_ERR_INVALID) == "invalid argument"
    assert "sm_103a" in L.bm_version()


def test_no_cpu_fallback_without_gpu(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes
    out = ctypes.c_void_p()
    st = L.lib.bm_context_create(0, None, ctypes.byref(out))
    assert st != L.BM_OK and not out.value
    assert L.bm_last_error() != ""


def test_library_is_built_for_sm_103a():
    # The build passes exactly one -gencode for compute_103a / sm_103a.
    from paper_2501_16122_gb300 import nvcc_build as b
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
