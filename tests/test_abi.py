"""The C ABI library builds, loads and exports every entry point that
include/mask.h declares; argument validation that happens before any CUDA
call is exercised on the host (no compute calls without a GPU)."""

import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2208_02734_gb300 import mask as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mask.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mask_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["mask_build", "mask_build_csr", "mask_query", "mask_query_csr", "mask_free",
              "mask_last_error", "mask_index_load", "mask_kmeans_assign",
              "mask_kmeans_update", "mask_kmeanspp"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = M.load()
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(M.EXPORTED) == _declared()


def test_exported_symbols_are_c_linkage():
    out = os.popen(f"nm -D --defined-only {M.library_path()}").read()
    syms = set(line.split()[-1] for line in out.splitlines() if line.strip())
    for name in _declared():
        assert name in syms, name


def _status(fn, *args):
    return fn(*args)


def test_build_rejects_bad_arguments_before_touching_the_gpu():
    lib = M.load()
    out = C.c_void_p()
    kp = (C.c_int32 * 2)(10, 20)  # level 1 larger than level 0
    X = np.zeros((100, 4), np.float32)
    assert lib.mask_build(X.ctypes.data, 100, 4, kp, 2, 5, 0, None, C.byref(out)) == M.MASK_EINVAL
    assert "k_per_level[1]" in M.mask_last_error()
    kp1 = (C.c_int32 * 1)(200)  # more centroids than points
    assert lib.mask_build(X.ctypes.data, 100, 4, kp1, 1, 5, 0, None, C.byref(out)) == M.MASK_EINVAL
    kp1 = (C.c_int32 * 1)(10)
    assert lib.mask_build(None, 100, 4, kp1, 1, 5, 0, None, C.byref(out)) == M.MASK_EINVAL
    assert lib.mask_build(X.ctypes.data, 0, 4, kp1, 1, 5, 0, None, C.byref(out)) == M.MASK_EINVAL
    assert lib.mask_build(X.ctypes.data, 100, 0, kp1, 1, 5, 0, None, C.byref(out)) == M.MASK_EINVAL
    assert lib.mask_build(X.ctypes.data, 100, 4, kp1, 0, 5, 0, None, C.byref(out)) == M.MASK_EINVAL
    assert lib.mask_build(X.ctypes.data, 100, 4, kp1, 1, -1, 0, None, C.byref(out)) == M.MASK_EINVAL
    assert lib.mask_build(X.ctypes.data, 100, 4, kp1, 1, 5, 0, None, None) == M.MASK_EINVAL


def test_query_rejects_null_index():
    lib = M.load()
    pr = (C.c_int32 * 1)(1)
    assert lib.mask_query(None, None, 1, 10, pr, 0, None, None, None) == M.MASK_EINVAL
    assert "NULL" in M.mask_last_error()


def test_binding_raises_mask_error():
    with pytest.raises(M.MaskError) as e:
        M.mask_build(np.zeros((5, 2), np.float32), [10], iters=1, seed=0)
    assert e.value.status == M.MASK_EINVAL


def test_free_of_null_is_a_no_op():
    M.load().mask_free(None)
