"""Pins of the oracle's multiword arithmetic against exact rationals.

Every L-limb operation of the oracle must return the exact result to within
a few units of 2^(-53 L) relative (Section 1: double double and quad double
arithmetic).  A dropped limb, a wrong sign or a lost error term changes the
error by a factor 2^53 or more and fails here.
"""

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1402_2626_gb300.inputs import cascade_from_fraction
from tests._util import ORACLE_OP_BOUND, cfr, fr

LS = (1, 2, 4)


def _rand_fraction(rng, spread=10):
    v = Fraction(float(rng.standard_normal()))
    for l in range(1, 6):
        v += Fraction(float(rng.standard_normal())) * Fraction(2) ** (-53 * l - int(rng.integers(0, 5)))
    return v * Fraction(2) ** int(rng.integers(-spread, spread + 1))


def _casc(v, L):
    return np.array(cascade_from_fraction(v, L))


def _rel(got: Fraction, want: Fraction) -> float:
    if want == 0:
        return float(abs(got))
    return abs(float((got - want) / want))


@pytest.mark.parametrize("L", LS)
def test_real_ops_exact(L):
    rng = np.random.default_rng(100 + L)
    bound = ORACLE_OP_BOUND[L]
    for _ in range(200):
        a, b = _rand_fraction(rng), _rand_fraction(rng)
        A, B = _casc(a, L), _casc(b, L)
        ea, eb = fr(A), fr(B)
        assert _rel(fr(oracle.real_op(L, "add", A, B)), ea + eb) <= bound * (abs(ea) + abs(eb)) / max(abs(ea + eb), Fraction(1, 10**300))
        assert _rel(fr(oracle.real_op(L, "sub", A, B)), ea - eb) <= bound * (abs(ea) + abs(eb)) / max(abs(ea - eb), Fraction(1, 10**300))
        assert _rel(fr(oracle.real_op(L, "mul", A, B)), ea * eb) <= bound
        assert _rel(fr(oracle.real_op(L, "div", A, B)), ea / eb) <= bound


@pytest.mark.parametrize("L", LS)
def test_sqrt_exact(L):
    rng = np.random.default_rng(200 + L)
    for _ in range(100):
        a = abs(_rand_fraction(rng))
        A = _casc(a, L)
        ea = fr(A)
        s = fr(oracle.real_op(L, "sqrt", A))
        # exact floor square root of ea at 400 fractional bits
        P = 400
        num = ea.numerator << (2 * P)
        root = Fraction(math.isqrt(num // ea.denominator * 1), 1) / Fraction(2) ** P
        # isqrt above is of floor(num/den); its error is far below 2^-300
        assert _rel(s, root) <= ORACLE_OP_BOUND[L]
    # perfect squares are exact
    for v in (4.0, 9.0, 0.25, 2.0 ** 60):
        got = oracle.real_op(L, "sqrt", _casc(Fraction(v), L))
        assert fr(got) == Fraction(math.sqrt(v))


@pytest.mark.parametrize("L", LS)
def test_cancellation_is_exact(L):
    # (1 + 2^-k) - 1 must give 2^-k exactly whenever 2^-k fits in L limbs
    for k in (10, 52, 60, 100, 150, 200):
        v = Fraction(1) + Fraction(1, 2 ** k)
        A = _casc(v, L)
        if fr(A) != v:
            continue
        d = oracle.real_op(L, "sub", A, _casc(Fraction(1), L))
        assert fr(d) == Fraction(1, 2 ** k)
    A = _casc(Fraction(1, 3), L)
    assert fr(oracle.real_op(L, "sub", A, A)) == 0


@pytest.mark.parametrize("L", LS)
def test_complex_ops_exact(L):
    rng = np.random.default_rng(300 + L)
    bound = ORACLE_OP_BOUND[L]
    for _ in range(100):
        ar, ai, br, bi = (_rand_fraction(rng, 3) for _ in range(4))
        A = np.stack([_casc(ar, L), _casc(ai, L)])
        B = np.stack([_casc(br, L), _casc(bi, L)])
        (ar, ai), (br, bi) = cfr(A), cfr(B)
        mag = (abs(ar) + abs(ai)) * (abs(br) + abs(bi))
        # product: each part within one rounding of the exact value
        c = cfr(oracle.cplx_op(L, "mul", A, B))
        assert abs(float(c[0] - (ar * br - ai * bi))) <= bound * float(mag)
        assert abs(float(c[1] - (ar * bi + ai * br))) <= bound * float(mag)
        # conjugated product (the inner products of Section 3)
        c = cfr(oracle.cplx_op(L, "conj_mul", A, B))
        assert abs(float(c[0] - (ar * br + ai * bi))) <= bound * float(mag)
        assert abs(float(c[1] - (ar * bi - ai * br))) <= bound * float(mag)
        # |a|^2
        c = cfr(oracle.cplx_op(L, "abs2", A))
        assert _rel(c[0], ar * ar + ai * ai) <= bound and c[1] == 0
        # a / real
        c = cfr(oracle.cplx_op(L, "div_real", A, B))
        assert _rel(c[0], ar / br) <= bound and _rel(c[1], ai / br) <= bound
        # sums
        c = cfr(oracle.cplx_op(L, "add", A, B))
        assert abs(float(c[0] - (ar + br))) <= bound * float(abs(ar) + abs(br))
        assert abs(float(c[1] - (ai + bi))) <= bound * float(abs(ai) + abs(bi))
