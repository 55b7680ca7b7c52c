"""Host-side pins of the block-floating-point integer products (csrc/ifx.cuh),
checked against Python's exact big integers."""

import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
MASK = (1 << 64) - 1


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("ifx") / "ifx_harness")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "ifx_harness.cu")],
                   check=True)
    return exe


def limbs(v, n):
    v &= (1 << (64 * n)) - 1
    return [(v >> (64 * i)) & MASK for i in range(n)]


def val(ls, signed=True):
    v = sum(x << (64 * i) for i, x in enumerate(ls))
    n = len(ls)
    if signed and v >> (64 * n - 1):
        v -= 1 << (64 * n)
    return v


def run(exe, lines):
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.strip().splitlines()
    return [[int(h, 16) for h in line.split()] for line in out]


def rand_signed(rng, K, bits=None):
    bits = bits if bits is not None else 64 * K - 2
    mag = int(rng.integers(0, 2 ** 62)) << max(bits - 62, 0)
    mag |= int.from_bytes(rng.bytes(8 * K), "little") & ((1 << max(bits - 62, 0)) - 1)
    mag &= (1 << bits) - 1
    return -mag if rng.random() < 0.5 else mag


@pytest.mark.parametrize("K", [1, 2, 4])
def test_mul_shift(harness, K):
    rng = np.random.default_rng(K)
    cases = []
    for _ in range(300):
        a = rand_signed(rng, K, int(rng.integers(1, 64 * K - 1)))
        b = rand_signed(rng, K, int(rng.integers(1, 64 * K - 1)))
        cases.append((a, b))
    cases += [(0, 5), (-(1 << (64 * K - 2)), 1 << (64 * K - 2)), (1, -1)]
    lines = [f"mul {K} " + " ".join("%x" % x for x in limbs(a, K) + limbs(b, K)) for a, b in cases]
    for (a, b), got in zip(cases, run(harness, lines)):
        exact = a * b
        want = abs(exact) >> (64 * K - 2)
        want = -want if exact < 0 else want
        g = val(got)
        slack = 1 if K < 4 else 2  # K = 4 leaves out the lowest partial products
        assert abs(g - want) <= slack, (K, a, b, g, want)


@pytest.mark.parametrize("K", [1, 2, 4])
def test_square_add_sub_sar_bitlen(harness, K):
    rng = np.random.default_rng(10 + K)
    lines, exp = [], []
    for _ in range(200):
        a = rand_signed(rng, K)
        b = rand_signed(rng, K)
        s = int(rng.integers(0, 64 * K))
        z = [0] * K
        lines.append(f"sq {K} " + " ".join("%x" % x for x in limbs(a, K) + z))
        exp.append(("sq", a * a))
        lines.append(f"add {K} " + " ".join("%x" % x for x in limbs(a, K) + limbs(b, K)))
        exp.append(("add", val(limbs(a + b, K))))
        lines.append(f"sub {K} " + " ".join("%x" % x for x in limbs(a, K) + limbs(b, K)))
        exp.append(("sub", val(limbs(a - b, K))))
        lines.append(f"sar {K} " + " ".join("%x" % x for x in limbs(a, K) + z) + f" {s}")
        exp.append(("sar", a >> s))
        lines.append(f"bitlen {K} " + " ".join("%x" % x for x in limbs(abs(a), K) + z))
        exp.append(("bitlen", abs(a).bit_length()))
    for (kind, want), got in zip(exp, run(harness, lines)):
        if kind == "sq":
            assert val(got, signed=False) == want
        elif kind == "bitlen":
            assert got[0] == want
        else:
            assert val(got) == want, kind


@pytest.mark.parametrize("K", [1, 2, 4])
def test_mul_full(harness, K):
    """ix_mul_full: exact signed (K+1)-limb x K-limb products."""
    rng = np.random.default_rng(70 + K)
    cases = [(rand_signed(rng, K + 1, 64 * K + 40), rand_signed(rng, K)) for _ in range(200)]
    cases += [(0, 5), (-1, -1), (-(1 << (64 * K + 40)), (1 << (64 * K - 2)) - 1)]
    lines = []
    for a, b in cases:
        la = limbs(a, K + 1)
        lines.append(f"mulf {K} " + " ".join("%x" % x for x in la[:K] + limbs(b, K) + la[K:]))
    for (a, b), got in zip(cases, run(harness, lines)):
        assert val(got) == a * b


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 9])
def test_barrel_shifts(harness, N):
    """ix_sar (arithmetic) and ix_shl (bits above 64 N lost) for every shift
    0 <= s < 64 N at the widths the kernels use (K, K+1, 2K+1, 3K+2 limbs)."""
    rng = np.random.default_rng(90 + N)
    lines, exp = [], []
    mod = 1 << (64 * N)
    shifts = list(range(0, 64 * N, 7 if N > 2 else 1)) + [64 * N - 1, 63, 64, 65]
    for s in shifts:
        if s >= 64 * N:
            continue
        a = rand_signed(rng, N)
        lines.append(f"xsar {N} " + " ".join("%x" % x for x in limbs(a, N)) + f" {s}")
        exp.append(a >> s)
        lines.append(f"xshl {N} " + " ".join("%x" % x for x in limbs(a, N)) + f" {s}")
        exp.append(val(limbs((a << s) % mod, N)))
    for want, got in zip(exp, run(harness, lines)):
        assert val(got) == want


@pytest.mark.parametrize("K", [1, 2, 4])
def test_rsqrt_frac(harness, K):
    """Y = 2^(64K-2)/sqrt(t) for t = tt/2^(64K) in [1/4, 1), to within a few units."""
    import math
    rng = np.random.default_rng(50 + K)
    ts = [1 << (64 * K - 2), (1 << (64 * K)) - 1]
    for _ in range(200):
        v = int.from_bytes(rng.bytes(8 * K), "little")
        ts.append((v >> 2) | (1 << (64 * K - 2)))
    lines = [f"rsqrt {K} " + " ".join("%x" % x for x in limbs(t, K) + [0] * K) for t in ts]
    S = 64 * K - 2
    for t, got in zip(ts, run(harness, lines)):
        Y = val(got, signed=False)
        # exact: floor(2^S * sqrt(2^(64K) / t)) = isqrt(2^(2S + 64K) // t)
        want = math.isqrt((1 << (2 * S + 64 * K)) // t)
        assert abs(Y - want) <= 8, (K, t, Y - want)


@pytest.mark.parametrize("K", [1, 2, 4])
def test_rsqrt_from_any_seed_within_ulps(harness, K):
    """The steps after the seed reach Y = 2^(64K-2)/sqrt(t) to within a few units
    from every FP32 seed within 8 ulp (2^-20) of 1/sqrt(t): the device's rsqrtf
    is within 2 ulp, the host's 1/sqrtf within 1."""
    import math
    rng = np.random.default_rng(90 + K)
    ts = [1 << (64 * K - 2), (1 << (64 * K)) - 1, (1 << (64 * K - 1)) + 1]
    for _ in range(150):
        v = int.from_bytes(rng.bytes(8 * K), "little")
        ts.append((v >> 2) | (1 << (64 * K - 2)))
    S = 64 * K - 2
    lines, want = [], []
    for t in ts:
        # y = 2^(32K)/sqrt(t) in (1, 2]; its 24-bit grid is y 2^23
        g = math.isqrt((1 << (64 * K + 46)) // t)
        exact = math.isqrt((1 << (2 * S + 64 * K)) // t)
        for m in (-8, -3, -2, -1, 0, 1, 2, 3, 8):
            seed = (g + m) << 39
            lines.append(f"rsqrtseed {K} " + " ".join("%x" % x for x in limbs(t, K) + [0] * K)
                         + " %x" % seed)
            want.append(exact)
    for w, got in zip(want, run(harness, lines)):
        Y = val(got, signed=False)
        assert abs(Y - w) <= 8, (K, Y - w)
