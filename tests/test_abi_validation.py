"""Argument validation of the C ABI, on the CPU: every call here is rejected
with BM_ERR_INVALID and a message before the library touches CUDA, so the
checks of include/bm.h's error contracts run without a GPU (the library is
loaded through the same binding the GPU tests use).  Also: without the
library every entry point raises (there is no fallback), and the package
imports nothing from the oracle."""
import ctypes
import math

import numpy as np
import pytest

from paper_2204_14067_gb300 import binding as B

INVALID = B.BM_ERR_INVALID


def _raises(fn, *args, match, **kw):
    with pytest.raises(B.BMError) as ei:
        fn(*args, **kw)
    assert ei.value.status == INVALID, ei.value
    assert match in str(ei.value), str(ei.value)


def _coo(nnz=3):
    return (np.arange(nnz, dtype=np.int32), np.arange(nnz, dtype=np.int32), np.ones(nnz, dtype=np.float32))


@pytest.mark.parametrize("m, n, lam, k_max, match", [
    (0, 5, 0.5, 1, "m and n must be >= 1"),
    (5, 5, 0.0, 1, "lambda must be finite and > 0"),
    (5, 5, math.nan, 1, "lambda must be finite and > 0"),
    (5, 5, math.inf, 1, "lambda must be finite and > 0"),
    (5, 5, 0.5, 0, "k_max must be in [1, min(m, n)]"),
    (5, 9, 0.5, 6, "k_max must be in [1, min(m, n)]"),
    (500, 500, 0.5, 128, "k_max must be in [1, min(m, n)]"),
])
def test_create_rejects_bad_sizes_and_lambda(m, n, lam, k_max, match):
    r, c, v = _coo()
    _raises(B.bm_create, m, n, r, c, v, lam, k_max, match=match)


@pytest.mark.parametrize("field, value, match", [
    ("alpha", 0.0, "alpha must be > 0"),
    ("lmsvd_p", 2, "lmsvd_p must be 0 or 1"),
    ("precision", 2, "precision must be 0 or 1"),
    ("step_rule", 3, "step_rule must be 0 or 1"),
    ("value_codec", -1, "value_codec must be 0 or 1"),
    ("bm_solver", 2, "bm_solver must be 0 or 1"),
    ("tensor_grams", 2, "tensor_grams must be 0 or 1"),
    ("lmsvd_imax", 0, "iteration counts out of range"),
])
def test_create_rejects_bad_options(field, value, match):
    o = B.bm_default_options()
    setattr(o, field, value)
    r, c, v = _coo()
    _raises(B.bm_create, 5, 5, r, c, v, 0.5, 2, o, match=match)


def test_create_rejects_null_arrays_and_null_output():
    L = B.lib()
    h = B._P()
    st = L.bm_create(5, 5, 3, None, None, None, 0.5, 2, None, ctypes.byref(h))
    assert st == INVALID and b"NULL index or value array" in L.bm_last_error(None)
    assert L.bm_create(5, 5, 0, None, None, None, 0.5, 2, None, None) == INVALID
    assert L.bm_default_options(None) == INVALID


@pytest.mark.parametrize("n, lam, k_max, match", [
    (1, -1.0, 1, "n must be in [2, 2^31)"),
    (10, math.nan, 2, "lambda must be finite"),
    (10, -1.0, 0, "k_max out of range"),
    (10, -1.0, 11, "k_max out of range"),
    (400, -1.0, 129, "k_max out of range"),
])
def test_distance_geometry_create_rejects_bad_arguments(n, lam, k_max, match):
    i = np.array([0, 1], np.int32)
    j = np.array([1, 2 % n], np.int32)
    d = np.ones(2, np.float32)
    _raises(B.bm_edm_create, n, i, j, d, lam, k_max, match=match)


def test_batch_and_server_reject_bad_arguments():
    _raises(B.bm_batch_create, [], match="need at least one handle")
    _raises(B.bm_server_create, max_active=0, match="max_active, max_outer >= 1")
    _raises(B.bm_server_create, precision=2, match="precision and keep_factors 0 or 1")
    _raises(B.bm_server_create, max_outer=0, match="max_active, max_outer >= 1")


@pytest.mark.parametrize("m, k, ld, lam, match", [
    (0, 4, 4, 0.5, "m and n must be >= 1"),
    (300_000, 4, 4, 0.5, "exceeds BM_NOALLOC_MAX_ROWS"),
    (10, 0, 4, 0.5, "need 1 <= k <= 128"),
    (10, 5, 6, 0.5, "ld % 4 == 0"),
    (10, 8, 4, 0.5, "k <= ld <= 128"),
    (10, 4, 4, math.inf, "lambda must be finite in FP32"),
    (10, 4, 4, 1e39, "lambda must be finite in FP32"),
])
def test_allocation_free_entry_rejects_bad_arguments(m, k, ld, lam, match):
    _raises(B.bm_loss_grad_csr_noalloc, m, 20, None, None, None, None, None, k, ld, lam, None, None, match=match)


@pytest.mark.parametrize("n, mode, match", [
    (0, 0, "need 1 <= n <= 256"),
    (257, 0, "need 1 <= n <= 256"),
    (4, 3, "mode must be 0, 1 or 2"),
])
def test_small_eigensolver_rejects_bad_arguments(n, mode, match):
    S = np.zeros((max(n, 1), max(n, 1)))
    L = B.lib()
    st = L.bm_sym_eig(S.ctypes.data, n, None, None, mode, None)
    assert st == INVALID
    assert match in L.bm_dense_last_error().decode()


def test_missing_library_fails_loudly(monkeypatch):
    """No fallback: without libbm.so every entry point raises."""
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", "/nonexistent/libbm.so")
    r, c, v = _coo()
    with pytest.raises(RuntimeError, match="is missing"):
        B.bm_create(5, 5, r, c, v, 0.5, 2)
    with pytest.raises(RuntimeError, match="is missing"):
        B.bm_default_options()


def test_package_never_imports_the_oracle():
    """The library's Python side is marshalling only: importing the package
    and loading the library pulls in no module of the oracle (checked in a
    fresh interpreter, as a user would run it)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; import paper_2204_14067_gb300 as P; P.lib(); P.bm_default_options(); "
            "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]; "
            "assert not bad, bad; print('clean')")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120, cwd=root)
    assert out.returncode == 0 and "clean" in out.stdout, out.stderr[-500:]
