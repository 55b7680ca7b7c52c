"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every function include/gn.h declares, and rejects malformed
systems (Section 1: sparse distributed form) before touching the device."""

import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1402_2626_gb300 import build, gn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gn.load_library()


def _declared():
    src = open(os.path.join(ROOT, "include", "gn.h")).read()
    return sorted(set(re.findall(r"\b(gn_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(gn.SYMBOLS)


def test_status_strings(lib):
    assert lib.gn_status_str(0) == b"ok"
    assert lib.gn_status_str(4) == b"singular Jacobian"
    assert lib.gn_version() >= 100


def _create(lib, N, n, poly_ptr, mono_ptr, var, exp, coef, limbs=1):
    pp = np.asarray(poly_ptr, np.int64)
    mp = np.asarray(mono_ptr, np.int64)
    v = np.asarray(var, np.int32)
    e = np.asarray(exp, np.uint8)
    c = np.asarray(coef, np.float64)
    h = C.c_void_p()
    return lib.gn_system_create(C.byref(h), N, n, len(mp) - 1,
                                pp.ctypes.data_as(C.POINTER(C.c_int64)),
                                mp.ctypes.data_as(C.POINTER(C.c_int64)),
                                v.ctypes.data_as(C.POINTER(C.c_int32)),
                                e.ctypes.data_as(C.POINTER(C.c_uint8)),
                                c.ctypes.data_as(C.POINTER(C.c_double)), limbs)


def test_rejects_malformed_systems(lib):
    coef = np.zeros((2, 2, 1))
    # N < n
    assert _create(lib, 1, 2, [0, 2], [0, 1, 2], [0, 1], [1, 1], coef) == 1
    # variable out of range
    assert _create(lib, 2, 2, [0, 1, 2], [0, 1, 2], [0, 2], [1, 1], coef) == 1
    # repeated variable in a monomial
    assert _create(lib, 2, 2, [0, 1, 2], [0, 2, 3], [1, 1, 0], [1, 1, 1], coef) == 1
    # exponent 0
    assert _create(lib, 2, 2, [0, 1, 2], [0, 1, 2], [0, 1], [0, 1], coef) == 1
    # pointers not monotone / not ending at T
    assert _create(lib, 2, 2, [0, 2, 1], [0, 1, 2], [0, 1], [1, 1], coef) == 1
    assert _create(lib, 2, 2, [0, 1, 3], [0, 1, 2], [0, 1], [1, 1], coef) == 1
    # bad limb count
    assert _create(lib, 2, 2, [0, 1, 2], [0, 1, 2], [0, 1], [1, 1], coef, limbs=3) == 1
    # null output handle
    assert lib.gn_system_create(None, 2, 2, 0, None, None, None, None, None, 1) == 1


def test_calls_reject_null_handles(lib):
    assert lib.gn_eval(None, 2, None, None, None, 0, None) == 1
    assert lib.gn_lstsq(None, 2, 4, 3, None, 4, None, None, None) == 1
    assert lib.gn_newton(None, 2, None, 1, 0.0, None, None) == 1
    assert lib.gn_system_destroy(None) == 1
    assert lib.gn_system_set_arith(None, 0) == 1
    assert lib.gn_mgs(None, 2, 4, 3, None, 4, None, None, None) == 1
    assert lib.gn_batch_newton(None, 2, None, 1, None, None, None) == 1
    assert lib.gn_batch_destroy(None) == 1
    assert lib.gn_batch_create(None, 1, None, 0, None, None, None, None, None, 1) == 1
    assert lib.gn_adjoint(None, 2, None, None, None, None, 0, None) == 1
    assert lib.gn_system_set_coef(None, None, 2, None) == 1
    assert lib.gn_newton_mixed(None, 4, None, 3, 4, 0.0, None, None) == 1
