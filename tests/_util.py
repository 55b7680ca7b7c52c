"""Shared test helpers: exact conversions, scales and tolerances.

No arithmetic of the method lives here: only conversions of limb arrays to
exact rationals, error measures and the tolerance table.
"""

from __future__ import annotations

from fractions import Fraction

import numpy as np

# Componentwise tolerances for GPU-vs-oracle parity, per precision (limbs).
# Errors are measured relative to the condition scale S of each entry
# (the sum of the magnitudes of the terms that make it up).
PARITY_TOL = {1: 1e-13, 2: 1e-26, 4: 1e-58}

# Bound on one rounded operation of the oracle's L-limb arithmetic.
ORACLE_OP_BOUND = {1: 2.0 ** -51, 2: 2.0 ** -104, 4: 2.0 ** -210}

NAMES = {1: "D", 2: "DD", 4: "QD"}


def fr(a) -> Fraction:
    """Exact value of a limb vector."""
    return sum((Fraction(float(v)) for v in np.asarray(a, dtype=np.float64).ravel()), Fraction(0))


def cfr(a):
    a = np.asarray(a, dtype=np.float64)
    return (fr(a[0]), fr(a[1]))


def cabs_f(z) -> float:
    re, im = z
    return float(abs(complex(float(re), float(im))))


def cdiff(a, b) -> float:
    """|a - b| for two exact complex pairs, as a float."""
    return cabs_f((a[0] - b[0], a[1] - b[1]))


def limb_sum(a) -> np.ndarray:
    """Sum of limbs as complex128 (leading ~53 bits), for scales only."""
    a = np.asarray(a, dtype=np.float64)
    return a[..., 0, :].sum(-1) + 1j * a[..., 1, :].sum(-1)


def limb_diff(a, b) -> np.ndarray:
    """|a - b| for limb arrays [..., 2, L], accurate even when a ~ b.

    Subtracts limb by limb from the leading limb down, using the fact that
    both cascades have nonoverlapping limbs: the difference is then formed in
    double-double-like accuracy, far below every tolerance used here.
    """
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = a - b  # per-limb differences (each exact up to one rounding)
    re = np.zeros(d.shape[:-2])
    im = np.zeros(d.shape[:-2])
    # sum from the smallest limb to the largest
    for l in range(d.shape[-1] - 1, -1, -1):
        re = re + d[..., 0, l]
        im = im + d[..., 1, l]
    return np.hypot(re, im)


def term_scales(system, x, rows=None):
    """Per-entry condition scales of f and J (double precision).

    S_f[i] = sum over the terms t of poly i of |c_t x^{a_t}|;
    S_J[i, v] = sum over the terms containing v of |d_tv c_t x^{a_t - e_v}|.
    """
    x = np.asarray(x)
    xc = x[:, 0, 0] + 1j * x[:, 1, 0]
    ax = np.abs(xc)
    r0, r1 = (0, system.N) if rows is None else rows
    Sf = np.zeros(r1 - r0)
    SJ = np.zeros((r1 - r0, system.n))
    cabs = np.abs(system.coef[:, 0, 0] + 1j * system.coef[:, 1, 0])
    for i in range(r0, r1):
        for t in range(int(system.poly_ptr[i]), int(system.poly_ptr[i + 1])):
            a, b = int(system.mono_ptr[t]), int(system.mono_ptr[t + 1])
            vs = system.var[a:b]
            ds = system.exp[a:b].astype(np.float64)
            mag = cabs[t] * np.prod(ax[vs] ** ds) if b > a else cabs[t]
            Sf[i - r0] += mag
            for v, d in zip(vs, ds):
                SJ[i - r0, v] += d * mag / ax[v]
    return Sf, SJ
