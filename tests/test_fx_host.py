"""Host-side pins of the integer fixed-point accumulator (csrc/fx.cuh).

The same source that the kernels use for exact sums is compiled for the host
(nvcc, no GPU needed) and checked against exact rational sums: the sum of
the addends, truncated below 2^-F per addend, converted to a cascade of L
doubles, each the double nearest to what the limbs before it leave over.
"""

import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("fx") / "fx_harness")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "fx_harness.cu")],
                   check=True)
    return exe


def _hex(d):
    return "%x" % struct.unpack("<Q", struct.pack("<d", d))[0]


def _unhex(h):
    return struct.unpack("<d", struct.pack("<Q", int(h, 16)))[0]


def _run(exe, jobs):
    inp = ""
    for NL, F, L, vals in jobs:
        inp += f"{NL} {F} {L} {len(vals)}\n" + " ".join(_hex(v) for v in vals) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    res = []
    for line in out.strip().splitlines():
        p = line.split()
        res.append((int(p[0]), [_unhex(h) for h in p[1:]]))
    return res


def _truncate(v: Fraction, F: int) -> Fraction:
    """What fx keeps of one addend: |v| * 2^F truncated to an integer."""
    scaled = abs(v) * Fraction(2) ** F
    t = scaled.numerator // scaled.denominator
    return Fraction(t if v >= 0 else -t) / Fraction(2) ** F


@pytest.mark.parametrize("NL,L,F", [(3, 2, 180), (5, 4, 300), (2, 1, 118), (3, 2, 150)])
def test_sums_exact(harness, NL, L, F):
    rng = np.random.default_rng(NL * 100 + F)
    jobs = []
    for trial in range(60):
        n = int(rng.integers(1, 200))
        scale = 2.0 ** int(rng.integers(-30, 0))
        vals = (rng.standard_normal(n) * scale * np.exp(rng.uniform(-40, 0, n))).tolist()
        if trial % 5 == 0:  # heavy cancellation
            vals = vals + [-v for v in vals[: n // 2]]
        if trial % 7 == 0:
            vals += [0.0, 5e-324]  # zero and a subnormal add nothing
        jobs.append((NL, F, L, vals))
    res = _run(harness, jobs)
    for (NL_, F_, L_, vals), (ok, out) in zip(jobs, res):
        assert ok == 1
        exact = sum((_truncate(Fraction(v), F_) for v in vals if abs(v) >= 2.0 ** -1022), Fraction(0))
        got = sum((Fraction(o) for o in out), Fraction(0))
        # the cascade is exact up to the rounding of its last limb
        assert abs(got - exact) <= abs(exact) * Fraction(2) ** (-53 * L_ + 1) + Fraction(2) ** -F_
        # limbs are nonoverlapping: each at most half an ulp of the one before
        for a, b in zip(out, out[1:]):
            assert b == 0 or abs(b) <= abs(a) * 2.0 ** -53
        # the leading limb is the double nearest to the whole value
        if exact != 0:
            assert abs(Fraction(out[0]) - exact) <= abs(Fraction(out[0])) * Fraction(2) ** -53 * (1 + Fraction(2) ** -50)


def test_overflow_reported(harness):
    (ok, _), = _run(harness, [(3, 180, 2, [2.0 ** 20])])
    assert ok == 0


def test_exact_cancellation_to_zero(harness):
    vals = [1.0, 2.0 ** -100, -1.0, -(2.0 ** -100)]
    (ok, out), = _run(harness, [(3, 180, 2, vals)])
    assert ok == 1 and out == [0.0, 0.0]
    (ok, out), = _run(harness, [(3, 180, 2, [1.0, 2.0 ** -100, -1.0])])
    assert out[0] == 2.0 ** -100 and out[1] == 0.0
