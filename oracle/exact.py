"""Exact-rational mode of the oracle (test infrastructure only).

Every input is a double (or a cascade of doubles), hence an exact dyadic
rational, so f, J and one Gauss-Newton step can be computed exactly on tiny
inputs with ``fractions.Fraction``:

* f_i(x) = sum_t c_t prod_j x_j^{d_tj} and
  J_iv(x) = sum_{t contains v} c_t d_tv x_v^{d_tv - 1} prod_{j != v} x_j^{d_tj}
  (Section 2, eq. 1 and Section 2.3: the plain definition);
* the least-squares step dx minimising ||J dx + f||_2 (Sections 3 and 4) from
  the normal equations (J^H J) dx = -J^H f, solved by exact Gaussian
  elimination.  For a J of full column rank this is the same vector the
  QR route of Section 3 reaches; it avoids the square roots of Gram-Schmidt,
  which are irrational.

Complex numbers are pairs (re, im) of Fractions.
"""

from __future__ import annotations

from fractions import Fraction

import numpy as np

ZERO = (Fraction(0), Fraction(0))
ONE = (Fraction(1), Fraction(0))


def cx(re, im=0.0):
    return (Fraction(re), Fraction(im))


def from_limbs(a) -> tuple:
    """Exact value of one complex entry [2, L] of doubles."""
    a = np.asarray(a, dtype=np.float64)
    return (sum((Fraction(float(v)) for v in a[0]), Fraction(0)),
            sum((Fraction(float(v)) for v in a[1]), Fraction(0)))


def add(a, b):
    return (a[0] + b[0], a[1] + b[1])


def sub(a, b):
    return (a[0] - b[0], a[1] - b[1])


def mul(a, b):
    return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])


def conj(a):
    return (a[0], -a[1])


def scale(a, s):
    s = Fraction(s)
    return (a[0] * s, a[1] * s)


def div(a, b):
    den = b[0] * b[0] + b[1] * b[1]
    num = mul(a, conj(b))
    return (num[0] / den, num[1] / den)


def power(a, d):
    r = ONE
    for _ in range(d):
        r = mul(r, a)
    return r


def evaluate(system, x, rows=None, L: int = 4):
    """Exact f (list) and J (dict (i, v) -> value) at x ([n, 2, >=1] doubles).

    Coefficients are taken with their first L limbs, as every precision-L
    computation reads them.
    """
    n = system.n
    xs = [from_limbs(np.asarray(x)[v]) for v in range(n)]
    r0, r1 = (0, system.N) if rows is None else rows
    coef = system.coef_limbs(L)
    f = []
    J = {}
    for i in range(r0, r1):
        fi = ZERO
        for t in range(int(system.poly_ptr[i]), int(system.poly_ptr[i + 1])):
            a, b = int(system.mono_ptr[t]), int(system.mono_ptr[t + 1])
            vs = [int(v) for v in system.var[a:b]]
            ds = [int(d) for d in system.exp[a:b]]
            c = from_limbs(coef[t])
            term = c
            for v, d in zip(vs, ds):
                term = mul(term, power(xs[v], d))
            fi = add(fi, term)
            for s, (v, d) in enumerate(zip(vs, ds)):
                p = scale(c, d)
                for r, (w, e) in enumerate(zip(vs, ds)):
                    p = mul(p, power(xs[w], e - 1 if r == s else e))
                J[(i, v)] = add(J.get((i, v), ZERO), p)
        f.append(fi)
    return f, J


def dense_jacobian(J, rows, n):
    r0, r1 = rows
    return [[J.get((i, v), ZERO) for v in range(n)] for i in range(r0, r1)]


def solve(Amat, bvec):
    """Exact Gaussian elimination with partial pivoting on nonzeros."""
    m = len(Amat)
    A = [list(row) + [bvec[i]] for i, row in enumerate(Amat)]
    for c in range(m):
        p = next((r for r in range(c, m) if A[r][c] != ZERO), None)
        if p is None:
            raise ZeroDivisionError("singular normal equations")
        A[c], A[p] = A[p], A[c]
        inv = div(ONE, A[c][c])
        for r in range(m):
            if r != c and A[r][c] != ZERO:
                fac = mul(A[r][c], inv)
                A[r] = [sub(A[r][j], mul(fac, A[c][j])) for j in range(m + 1)]
    return [mul(A[i][m], div(ONE, A[i][i])) for i in range(m)]


def lstsq_step(system, x, L: int = 4):
    """Exact Gauss-Newton step dx: (J^H J) dx = -J^H f (Section 4)."""
    n, N = system.n, system.N
    f, J = evaluate(system, x, L=L)
    Jd = dense_jacobian(J, (0, N), n)
    G = [[ZERO] * n for _ in range(n)]
    g = [ZERO] * n
    for a in range(n):
        for b in range(n):
            s = ZERO
            for i in range(N):
                s = add(s, mul(conj(Jd[i][a]), Jd[i][b]))
            G[a][b] = s
        s = ZERO
        for i in range(N):
            s = sub(s, mul(conj(Jd[i][a]), f[i]))
        g[a] = s
    return solve(G, g)


def to_float(a) -> complex:
    return complex(float(a[0]), float(a[1]))
