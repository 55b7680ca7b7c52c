"""The paper's benchmark systems (Section 5): their generators, and the
oracle's evaluation and Newton's method on them, pinned to closed forms and to
computations independent of the oracle.

* Cyclic n-roots (Section 5.3, eq. 7): n^2 - n + 2 monomials; at x = 1 every
  polynomial i < n is n and every Jacobian entry of row i is i (variable v
  lies in i of the n windows of length i); at x = -1 the signs follow the
  degrees; for odd n the point x_k = w^k (w = exp(2 pi i / n)) is a root.
* The Newton homotopy f(x) - t f(z) of Section 5.3: at x = z the residual is
  exactly (1 - t) f(z).
* The Chandrasekhar H-equation (Section 5.2, eq. 6): at H = 1,
  f_i = -c sum_j i / (i + j) exactly; Newton's method from H = 1 converges
  quadratically to the root that the fixed-point form
  H_i = 1 / (1 - c / (2n) sum_j i/(i+j) H_j) gives in 80-digit arithmetic.
"""

from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1402_2626_gb300 import inputs
from tests._util import ORACLE_OP_BOUND, PARITY_TOL, cdiff, cfr, limb_diff


def _const_point(n, re, L):
    x = np.zeros((n, 2, L))
    x[:, 0, 0] = re
    return x


@pytest.mark.parametrize("n", [5, 8, 70])
def test_cyclic_structure(n):
    s = inputs.cyclic(n)
    assert s.N == s.n == n and s.T == n * n - n + 2
    for i in range(n - 1):
        t0, t1 = int(s.poly_ptr[i]), int(s.poly_ptr[i + 1])
        assert t1 - t0 == n
        sups = set()
        for t in range(t0, t1):
            a, b = int(s.mono_ptr[t]), int(s.mono_ptr[t + 1])
            assert b - a == i + 1 and np.all(s.exp[a:b] == 1)
            sups.add(tuple(s.var[a:b]))
        assert len(sups) == n or i + 1 == n  # distinct windows
    t0 = int(s.poly_ptr[n - 1])
    assert int(s.mono_ptr[t0 + 1] - s.mono_ptr[t0]) == n and s.coef[t0 + 1, 0, 0] == -1.0


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("n,mode", [(6, "definition"), (33, "definition"), (6, "reverse"),
                                    (70, "reverse")])
def test_cyclic_at_plus_minus_one(n, mode, L):
    s = inputs.cyclic(n)
    for sign in (1.0, -1.0):
        f, J, _ = oracle.evaluate(s, _const_point(n, sign, L), L, mode)
        for i in range(n - 1):
            deg = i + 1
            assert cfr(f[i]) == (Fraction(n) * int(sign) ** deg, 0)
            want = Fraction(deg) * int(sign) ** (deg - 1)
            assert all(cfr(J[i, v]) == (want, 0) for v in range(n))
        assert cfr(f[n - 1]) == (Fraction(int(sign) ** n - 1), 0)
        assert all(cfr(J[n - 1, v]) == (Fraction(int(sign) ** (n - 1)), 0) for v in range(n))


@pytest.mark.parametrize("n", [5, 7, 65])
def test_cyclic_roots_of_unity(n):
    """x_k = w^k, w = exp(2 pi i / n), n odd, solves the cyclic n-roots
    system: f_i = w^(i(i-1)/2) sum_j w^(ij) = 0 for i < n, and the product
    of all w^k is w^(n(n-1)/2) = 1."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 80
    s = inputs.cyclic(n)
    L = 2
    x = np.zeros((n, 2, L))
    for k in range(n):
        z = mpmath.exp(2j * mpmath.pi * k / n)
        for part, v in enumerate((z.real, z.imag)):
            d0 = float(v)
            x[k, part] = (d0, float(v - d0))
    f, _, _ = oracle.evaluate(s, x, L)
    # each f_i sums n terms of modulus 1: rounding of about n u_DD
    assert np.abs(oracle.to_complex(f)).max() <= 1e3 * n * ORACLE_OP_BOUND[L]


def test_cyclic_homotopy_residual_at_z():
    n = 40
    t = 1.0 - 2.0 ** -20
    s = inputs.cyclic_homotopy(n, t=t, seed=3)
    z = s.x0[:, 0] + 1j * s.x0[:, 1]
    assert set(np.round(z, 12).tolist()) <= {1, 1j, -1, -1j}
    fz = []
    for i in range(1, n):
        fz.append(sum(np.prod(z[[(j + r) % n for r in range(i)]]) for j in range(n)))
    fz.append(np.prod(z) - 1)
    f, _, _ = oracle.evaluate(s, s.point("x0", 4), 4, jacobian=False)
    for i in range(n):
        want = (Fraction(1) - Fraction(t)) * Fraction(int(round(fz[i].real)))
        wanti = (Fraction(1) - Fraction(t)) * Fraction(int(round(fz[i].imag)))
        assert cfr(f[i]) == (want, wanti)


@pytest.mark.parametrize("L", [2, 4])
def test_chandrasekhar_at_one(L):
    n = 9
    c = Fraction(33, 64)
    s = inputs.chandrasekhar(n, c)
    f, _, _ = oracle.evaluate(s, s.point("x0", L), L, jacobian=False)
    for i in range(1, n + 1):
        want = -c * sum(Fraction(i, i + j) for j in range(1, n + 1))
        assert cdiff(cfr(f[i - 1]), (want, Fraction(0))) <= 4 * n * ORACLE_OP_BOUND[L] * 2 * n


def _chandra_fixed_point(n, c, digits=80, iters=400):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = digits
    cc = mpmath.mpf(c.numerator) / c.denominator
    H = [mpmath.mpf(1)] * n
    for _ in range(iters):
        H = [1 / (1 - cc / (2 * n) * sum(mpmath.mpf(i) / (i + j) * H[j - 1] for j in range(1, n + 1)))
             for i in range(1, n + 1)]
    return H


@pytest.mark.parametrize("n", [6, 16])
def test_chandrasekhar_newton_root(n):
    c = Fraction(33, 64)
    s = inputs.chandrasekhar(n, c)
    H = _chandra_fixed_point(n, c)
    for L, steps in ((2, 6), (4, 7)):
        x, hist = oracle.newton(s, s.point("x0", L), L, steps)
        ref = np.zeros((n, 2, L))
        for v in range(n):
            d0 = float(H[v])
            rest = H[v] - d0
            ref[v, 0, 0] = d0
            if L > 1:
                d1 = float(rest)
                ref[v, 0, 1] = d1
                if L > 2:
                    d2 = float(rest - d1)
                    ref[v, 0, 2] = d2
                    ref[v, 0, 3] = float(rest - d1 - d2)
        assert limb_diff(x, ref).max() <= PARITY_TOL[L], L
        # quadratic convergence from H = 1
        dx = [h[1] for h in hist]
        for a, b in zip(dx, dx[1:]):
            if a > 1e-12:
                assert b <= 10 * a * a, dx
