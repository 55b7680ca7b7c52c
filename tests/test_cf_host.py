"""Host-side pins of the integer-mantissa complex arithmetic (csrc/cf.cuh)
against exact rationals: products, small-integer scalings and conversions
are within a few units of 2^(-64K) of the exact result (normwise), well
inside one rounding of the L-limb format they stand in for."""

import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

from paper_1402_2626_gb300.inputs import cascade_from_fraction

HERE = os.path.dirname(os.path.abspath(__file__))
KL = [(1, 1), (2, 2), (4, 4)]
BOUND = {1: 2.0 ** -53, 2: 2.0 ** -106, 4: 2.0 ** -212}  # one unit of the L-limb format


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("cf") / "cf_harness")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "cf_harness.cu")],
                   check=True)
    return exe


def hx(d):
    return "%x" % struct.unpack("<Q", struct.pack("<d", d))[0]


def unhx(h):
    return struct.unpack("<d", struct.pack("<Q", int(h, 16)))[0]


def rnd(rng, L, spread=20):
    v = Fraction(float(rng.standard_normal()))
    for l in range(1, L + 2):
        v += Fraction(float(rng.standard_normal())) * Fraction(2) ** (-53 * l)
    return v * Fraction(2) ** int(rng.integers(-spread, spread + 1))


def run(exe, lines):
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.strip().splitlines()
    return [[unhx(h) for h in line.split()] for line in out]


def cval(limbs, L):
    re = sum((Fraction(x) for x in limbs[:L]), Fraction(0))
    im = sum((Fraction(x) for x in limbs[L:]), Fraction(0))
    return re, im


def cabs(re, im):
    return abs(complex(float(re), float(im)))


@pytest.mark.parametrize("K,L", KL)
def test_products(harness, K, L):
    rng = np.random.default_rng(K)
    cases, lines = [], []
    for t in range(150):
        a = (rnd(rng, L), rnd(rng, L))
        b = (rnd(rng, L), rnd(rng, L))
        if t % 10 == 0:
            a = (a[0], Fraction(0))  # real operand
        if t % 15 == 0:
            b = (b[0], -b[0] * (1 + Fraction(1, 2 ** 70)))  # cancellation in the product
        A = [cascade_from_fraction(a[0], L), cascade_from_fraction(a[1], L)]
        B = [cascade_from_fraction(b[0], L), cascade_from_fraction(b[1], L)]
        cases.append((cval(A[0] + A[1], L), cval(B[0] + B[1], L)))
        lines.append(f"mul {K} {L} " + " ".join(hx(x) for x in A[0] + A[1] + B[0] + B[1]))
    for ((ar, ai), (br, bi)), got in zip(cases, run(harness, lines)):
        er, ei = ar * br - ai * bi, ar * bi + ai * br
        gr, gi = cval(got, L)
        err = cabs(gr - er, gi - ei)
        assert err <= 16 * BOUND[L] * cabs(ar, ai) * cabs(br, bi), (K, err)


@pytest.mark.parametrize("K,L", KL)
def test_scale_and_round_trip(harness, K, L):
    rng = np.random.default_rng(10 + K)
    cases, lines = [], []
    for _ in range(100):
        a = (rnd(rng, L), rnd(rng, L))
        A = [cascade_from_fraction(a[0], L), cascade_from_fraction(a[1], L)]
        d = int(rng.integers(1, 256))
        av = cval(A[0] + A[1], L)
        cases.append(("scale", av, d))
        lines.append(f"scale {K} {L} " + " ".join(hx(x) for x in A[0] + A[1]) + f" {d}")
        cases.append(("rt", av, 1))
        lines.append(f"rt {K} {L} " + " ".join(hx(x) for x in A[0] + A[1]))
    lines.append(f"rt {K} {L} " + " ".join(hx(0.0) for _ in range(2 * L)))
    cases.append(("rt", (Fraction(0), Fraction(0)), 1))
    for (kind, (ar, ai), d), got in zip(cases, run(harness, lines)):
        gr, gi = cval(got, L)
        err = cabs(gr - d * ar, gi - d * ai)
        assert err <= 8 * BOUND[L] * d * cabs(ar, ai) + (0 if ar or ai else 0), (kind, K, err)


@pytest.mark.parametrize("K", [1, 2, 4])
def test_fast_forms_bit_identical(harness, K):
    """The renormalisation (one bit length of |re| | |im|, a branch-free shift for
    shifts of -8..55 bits) and the product (each part as one addition with a
    conditional complement and one conditional negation) equal, bit for bit,
    their written-out forms: separate left and right barrel shifts, and four
    signed truncated products added and subtracted."""
    n = 100000 if K < 4 else 50000
    out = subprocess.run([harness], input=f"same {K} {n} {1234567 + K}\n", capture_output=True,
                         text=True, check=True).stdout.split()
    assert out == ["ok", str(n)], out
