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


def lstsq_sensitivity(A, Ro):
    """First-order perturbation factors of one least-squares case.

    Both sides of a parity test run modified Gram-Schmidt, which is backward
    stable: each result is the exact factorisation of [A b] moved by a
    relative amount of order u_L, far below the stated tolerance tol_L.  The
    difference of the two results therefore obeys the standard first-order
    perturbation bounds with eps = tol_L, with the condition number kappa of
    A = [A b][:, :n] read from the oracle's R (same singular values as A):

      column j of R (b's column included):  |dr_kj| <= eps kappa ||a_j||
      column k < n of Q:                    |dq_ik| <= eps kappa
      solution x of min ||A x - b||:
          ||dx|| <= eps kappa (||x|| + (||b|| + kappa ||r||) / sigma_max)

    (R and Q: the sensitivity of the QR factors; x: the Golub-Van Loan /
    Wedin bound for least squares, r = b - A x, ||r|| = r_nn from MGS).
    Returns (kappa, column norms of [A b], the factor of eps for x).
    """
    A = np.asarray(A, dtype=np.float64)
    Ro = np.asarray(Ro, dtype=np.float64)
    n = Ro.shape[0] - 1
    cn = np.sqrt((A[..., 0] ** 2).sum(axis=(0, 2)))  # ||a_j|| (double, leading limbs)
    Rc = Ro[:n, :n, 0, 0] + 1j * Ro[:n, :n, 1, 0]
    sv = np.linalg.svd(Rc, compute_uv=False)
    kappa = float(sv[0] / sv[-1])
    y = Ro[:n, n, 0, 0] + 1j * Ro[:n, n, 1, 0]
    x = np.linalg.solve(np.triu(Rc), y)
    rnorm = float(abs(Ro[n, n, 0, 0] + 1j * Ro[n, n, 1, 0]))
    fx = kappa * (float(np.linalg.norm(x)) + (float(cn[n]) + kappa * rnorm) / float(sv[0]))
    return kappa, cn, fx


def rounding_residual_scale(system, x, rows=None):
    """Per-row scale of |f_i(x)| at a computed root x.

    A root carried to relative accuracy eps in each component leaves, to
    first order, |f_i(x)| <= eps (S_f[i] + sum_v S_J[i, v] |x_v|): the
    evaluation's own rounding (S_f) plus the change of f under a relative
    move eps |x_v| of each variable (S_J the Jacobian's term scales).
    """
    Sf, SJ = term_scales(system, x, rows=rows)
    x = np.asarray(x)
    ax = np.abs(x[:, 0, 0] + 1j * x[:, 1, 0])
    return Sf + SJ @ ax
