"""Host-side pins of the batch generator (inputs.random_batch) and of the
batch boundary's validation: structure of every system, the exact root, and
independence of each system's random stream."""

import ctypes as C
from fractions import Fraction

import numpy as np
import pytest

from paper_1402_2626_gb300 import inputs


@pytest.fixture(scope="module")
def batch():
    return inputs.random_batch(24, 12345, n_range=(16, 40))


def test_structure(batch):
    b = batch
    assert b.sys_poly.tolist() == b.sys_var.tolist()  # square systems
    n = b.n
    assert np.all((n >= 16) & (n <= 40))
    for s in range(b.S):
        sy = b.system(s)
        assert sy.N == sy.n == n[s]
        assert sy.poly_ptr[0] == 0 and sy.poly_ptr[-1] == sy.T
        for i in range(sy.N):
            t0, t1 = int(sy.poly_ptr[i]), int(sy.poly_ptr[i + 1])
            M = t1 - t0 - 1  # the last term is the constant
            assert int(np.ceil(0.5 * sy.n)) <= M <= int(np.floor(2.0 * sy.n))
            assert sy.mono_ptr[t1] == sy.mono_ptr[t1 - 1]  # constant: empty support
            keys = set()
            for t in range(t0, t1 - 1):
                a, c = int(sy.mono_ptr[t]), int(sy.mono_ptr[t + 1])
                v, e = sy.var[a:c], sy.exp[a:c]
                assert 2 <= c - a <= min(16, sy.n)
                assert np.all(np.diff(v) > 0) and v.min() >= 0 and v.max() < sy.n
                assert np.all((e >= 1) & (e <= 4))
                assert np.hypot(*sy.coef[t, :, 0]) == pytest.approx(1.0, abs=1e-15)
                assert not np.any(sy.coef[t, :, 1:])
                keys.add((v.tobytes(), e.tobytes()))
            assert len(keys) == M  # distinct monomials within a polynomial


def test_exact_root(batch):
    """f(x*) = 0 up to the rounding of the constant term (4 limbs), checked
    with exact rationals: x*_j is a power of i, so every term is exact."""
    for s in (0, 7, 23):
        sy = batch.system(s)
        xs = [(Fraction(a), Fraction(b)) for a, b in sy.xstar]
        for i in range(sy.N):
            re = im = Fraction(0)
            for t in range(int(sy.poly_ptr[i]), int(sy.poly_ptr[i + 1])):
                cr = sum(Fraction(v) for v in sy.coef[t, 0])
                ci = sum(Fraction(v) for v in sy.coef[t, 1])
                for o in range(int(sy.mono_ptr[t]), int(sy.mono_ptr[t + 1])):
                    xr, xi = xs[sy.var[o]]
                    for _ in range(int(sy.exp[o])):
                        cr, ci = cr * xr - ci * xi, cr * xi + ci * xr
                re += cr
                im += ci
            assert abs(re) <= Fraction(1, 2 ** 200) and abs(im) <= Fraction(1, 2 ** 200)
        assert set(np.round(np.abs(sy.xstar).sum(axis=1), 12).tolist()) == {1.0}
        d = sy.x0 - sy.xstar
        assert np.allclose(np.hypot(d[:, 0], d[:, 1]), 1e-6, rtol=1e-9)


def test_system_streams_are_independent():
    a = inputs.random_batch(6, 99, n_range=(16, 24))
    b = inputs.random_batch(10, 99, n_range=(16, 24))
    for s in range(6):
        x, y = a.system(s), b.system(s)
        assert np.array_equal(x.var, y.var) and np.array_equal(x.coef, y.coef)
        assert np.array_equal(x.xstar, y.xstar)


def test_batch_create_rejects_malformed():
    from paper_1402_2626_gb300 import build, gn

    build.build()
    lib = gn.load_library()
    b = inputs.random_batch(2, 5, n_range=(16, 16))

    def create(var):
        h = C.c_void_p()
        ns = np.diff(b.sys_var).astype(np.int64)
        pp, mp = b.poly_ptr.astype(np.int64), b.mono_ptr.astype(np.int64)
        ex, cf = b.exp.astype(np.uint8), np.ascontiguousarray(b.coef[:, :, :1])
        return lib.gn_batch_create(C.byref(h), b.S, ns.ctypes.data_as(C.POINTER(C.c_int64)), b.T,
                                   pp.ctypes.data_as(C.POINTER(C.c_int64)),
                                   mp.ctypes.data_as(C.POINTER(C.c_int64)),
                                   var.ctypes.data_as(C.POINTER(C.c_int32)),
                                   ex.ctypes.data_as(C.POINTER(C.c_uint8)),
                                   cf.ctypes.data_as(C.POINTER(C.c_double)), 1)

    bad = b.var.astype(np.int32).copy()
    bad[5] = 16  # a local variable index out of its system's range
    assert create(bad) == 1
    bad = b.var.astype(np.int32).copy()
    bad[1] = bad[0]  # a repeated variable inside a monomial
    assert create(bad) == 1
