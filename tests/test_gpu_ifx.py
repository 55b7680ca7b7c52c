"""Device builds of the multi-limb integer operations (csrc/ifx.cuh) against
exact big-integer arithmetic and the host builds, bit for bit: the unsigned
product (with the K = 4 rule of partial products left out) on carry-heavy
operands, the signed shifted product, the square, and the reciprocal square
root from the device's FP32 seed."""

import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from tests.test_ifx_host import harness, limbs, rand_signed, run, val  # noqa: F401

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def gpu_harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path_factory.mktemp("ifxg") / "ifx_gpu_harness")
    subprocess.run([nvcc, "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe,
                    os.path.join(HERE, "ifx_gpu_harness.cu")], check=True)
    return exe


def umul_exact(a, b, K):
    """ix_umul's sum: every 64-bit partial product, except i + j < 2 for K = 4."""
    M = (1 << 64) - 1
    s = 0
    for i in range(K):
        for j in range(K):
            if K == 4 and i + j < 2:
                continue
            s += ((a >> (64 * i)) & M) * ((b >> (64 * j)) & M) << (64 * (i + j))
    return s


def special(K):
    top = (1 << (64 * K)) - 1
    return [0, 1, top, top - 1, 1 << (64 * K - 1), (1 << (64 * K - 1)) - 1, 1 << 63, (1 << 64) - 1,
            (1 << 32) - 1, int("f" * 8 + "0" * 8, 16) * sum(1 << (64 * i) for i in range(K))]


@pytest.mark.parametrize("K", [1, 2, 4])
def test_device_products_bit_exact(gpu_harness, harness, K):  # noqa: F811
    rng = np.random.default_rng(400 + K)
    us = special(K) + [int.from_bytes(rng.bytes(8 * K), "little") for _ in range(300)]
    pairs = [(a, b) for a in special(K) for b in special(K)]
    pairs += [(us[i], us[-1 - i]) for i in range(len(us))]
    lines = [f"umul {K} " + " ".join("%x" % x for x in limbs(a, K) + limbs(b, K)) for a, b in pairs]
    got = run(gpu_harness, lines)
    for (a, b), g in zip(pairs, got):
        assert val(g, signed=False) == umul_exact(a, b, K), (K, hex(a), hex(b))
    # the signed shifted product and the square: the device equals the host
    sg = [(rand_signed(rng, K), rand_signed(rng, K)) for _ in range(300)]
    sg += [(-(1 << (64 * K - 2)), 1 << (64 * K - 2)), (-(1 << (64 * K - 2)), -(1 << (64 * K - 2))),
           (0, 5), (-1, 1), ((1 << (64 * K - 2)) - 1, -((1 << (64 * K - 2)) - 1))]
    lines = [f"mul {K} " + " ".join("%x" % x for x in limbs(a, K) + limbs(b, K)) for a, b in sg]
    lines += [f"sq {K} " + " ".join("%x" % x for x in limbs(a, K) + [0] * K) for a, _ in sg]
    dev = run(gpu_harness, lines)
    host = run(harness, lines)
    assert dev == host
    for (a, _), g in zip(sg, dev[len(sg):]):
        assert val(g, signed=False) == a * a


@pytest.mark.parametrize("K", [1, 2, 4])
def test_device_rsqrt(gpu_harness, K):
    """From the device's rsqrtf seed: within 8 units of 2^(64K-2)/sqrt(t)."""
    rng = np.random.default_rng(500 + K)
    ts = [1 << (64 * K - 2), (1 << (64 * K)) - 1, (1 << (64 * K - 1)) + 1]
    for _ in range(500):
        v = int.from_bytes(rng.bytes(8 * K), "little")
        ts.append((v >> 2) | (1 << (64 * K - 2)))
    lines = [f"rsqrt {K} " + " ".join("%x" % x for x in limbs(t, K) + [0] * K) for t in ts]
    S = 64 * K - 2
    for t, g in zip(ts, run(gpu_harness, lines)):
        want = math.isqrt((1 << (2 * S + 64 * K)) // t)
        assert abs(val(g, signed=False) - want) <= 8, (K, t)
