"""Pins of the oracle's coefficient gradient (the adjoint of the Newton fixed point).

At a root x of f(x; c) = 0 the root moves with the coefficients by
dx = -J^+ (df/dc) dc, and a real loss with gradient g = dL/dRe x + i dL/dIm x
has the coefficient gradient sum_j g_j conj(dx_j / dc).  The oracle takes the
reverse route (R^H w = g, lambda = Q w, grad_t = -lambda_i conj(x^{a_t})).
The pins reach the same numbers by other routes:

* forward mode in exact rationals on tiny systems, square and overdetermined:
  for every coefficient c_t of polynomial i, v = dx/dc_t solves
  (J^H J) v = -J^H e_i x^{a_t} exactly, and grad_t = sum_j g_j conj(v_j);
* central finite differences in quad double: Re c_t and Im c_t are moved by
  +-h, Newton's method (Section 4) finds the moved root again, and
  (L(+h) - L(-h)) / 2h must match the real and the imaginary part of grad_t.
  This pins the formula itself (signs, conjugations, the polynomial a term
  belongs to), not only the linear algebra;
* a closed form: f(x) = c1 x + c0 has the root x = -c0/c1, so for
  L = |x|^2 the gradients are -2|x|^2 / conj(c1) and -2x / conj(c1).
"""

import dataclasses
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_1402_2626_gb300 import inputs
from paper_1402_2626_gb300.inputs import System
from tests._util import ORACLE_OP_BOUND, cdiff, cfr


def _exact_grad(s, x, g, L):
    """Forward-mode gradient of every coefficient, in exact rationals."""
    n, N = s.n, s.N
    _, Jd = exact.evaluate(s, x, L=L)
    J = exact.dense_jacobian(Jd, (0, N), n)
    G = [[exact.ZERO] * n for _ in range(n)]
    for a in range(n):
        for b in range(n):
            acc = exact.ZERO
            for i in range(N):
                acc = exact.add(acc, exact.mul(exact.conj(J[i][a]), J[i][b]))
            G[a][b] = acc
    xs = [exact.from_limbs(np.asarray(x)[v]) for v in range(n)]
    gs = [exact.from_limbs(np.asarray(g)[v]) for v in range(n)]
    out = []
    for i in range(N):
        for t in range(int(s.poly_ptr[i]), int(s.poly_ptr[i + 1])):
            a, b = int(s.mono_ptr[t]), int(s.mono_ptr[t + 1])
            m = exact.ONE
            for v, d in zip(s.var[a:b], s.exp[a:b]):
                m = exact.mul(m, exact.power(xs[int(v)], int(d)))
            # the column df/dc_t = e_i m; right-hand side -J^H e_i m
            rhs = [exact.sub(exact.ZERO, exact.mul(exact.conj(J[i][c]), m)) for c in range(n)]
            v = exact.solve(G, rhs)
            acc = exact.ZERO
            for j in range(n):
                acc = exact.add(acc, exact.mul(gs[j], exact.conj(v[j])))
            out.append(acc)
    return out


TINY = [
    ("square", dict(N=3, n=3, M=(2, 3), k=(1, 3), dmax=3, seed=11)),
    ("overdetermined", dict(N=5, n=3, M=(2, 3), k=(1, 3), dmax=3, seed=12)),
]


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("name,kw", TINY, ids=[t[0] for t in TINY])
def test_gradient_matches_exact_forward_mode(name, kw, L):
    s = inputs.random_system(kw["N"], kw["n"], kw["M"], kw["k"], kw["dmax"], seed=kw["seed"])
    x = s.point("xstar", L)
    g = 2.0 * x  # L = sum |x_j|^2; doubling is exact
    grad, _ = oracle.adjoint(s, x, g, L)
    ge = _exact_grad(s, x, g, L)
    scale = max(abs(exact.to_float(v)) for v in ge)
    assert scale > 0.1
    # a few dozen rounded operations on well-conditioned tiny J: the observed
    # error is about one rounding of the largest gradient; 100 leave headroom
    bound = 100 * ORACLE_OP_BOUND[L] * scale
    errs = [cdiff(cfr(grad[t]), ge[t]) for t in range(s.T)]
    assert max(errs) <= bound, (max(errs), bound)


def _loss_exact(x):
    return sum((cfr(x[v])[0] ** 2 + cfr(x[v])[1] ** 2 for v in range(x.shape[0])), Fraction(0))


def _moved(s, t, part, h):
    """Copy of s with Re (part 0) or Im (part 1) of coefficient t moved by h,
    kept as the nearest 4-limb cascade of the exact sum."""
    coef = s.coef.copy()
    val = sum((Fraction(float(v)) for v in coef[t, part]), Fraction(0)) + h
    coef[t, part, :] = inputs.cascade_from_fraction(val, 4)
    return dataclasses.replace(s, coef=coef)


FD_CASES = [
    ("square", dict(N=6, n=6, M=(3, 6), k=(1, 3), dmax=3, seed=21)),
    ("overdetermined", dict(N=8, n=5, M=(3, 5), k=(1, 3), dmax=3, seed=22)),
]


@pytest.mark.parametrize("name,kw", FD_CASES, ids=[c[0] for c in FD_CASES])
def test_gradient_matches_central_differences_qd(name, kw):
    s = inputs.random_system(kw["N"], kw["n"], kw["M"], kw["k"], kw["dmax"], seed=kw["seed"])
    L = 4
    x0, _ = oracle.newton(s, s.point("xstar", L), L, 2)  # the root of the stored system
    grad4, _ = oracle.adjoint(s, x0, 2.0 * x0, L)
    grad2, _ = oracle.adjoint(s, x0, 2.0 * x0, 2)
    h = Fraction(1, 2 ** 66)
    # every polynomial's first term, the last term and one constant term
    ts = sorted({int(s.poly_ptr[i]) for i in range(s.N)} | {s.T - 1, int(s.poly_ptr[1]) - 1})
    scale = float(np.abs(oracle.to_complex(grad4)).max())
    for t in ts:
        for part in (0, 1):
            lp = _loss_exact(oracle.newton(_moved(s, t, part, h), x0, L, 3)[0])
            lm = _loss_exact(oracle.newton(_moved(s, t, part, -h), x0, L, 3)[0])
            fd = (lp - lm) / (2 * h)
            # truncation ~ h^2 = 1e-40, the roots' rounding / h ~ 1e-43; the
            # DD gradient carries its own rounding, ~1e-32
            assert abs(float(fd - cfr(grad4[t])[part])) <= 1e-38 * scale, (t, part)
            assert abs(float(fd - cfr(grad2[t])[part])) <= 1e-30 * scale, (t, part)


@pytest.mark.parametrize("L", [1, 2, 4])
def test_closed_form_linear(L):
    # f(x) = (1 + 2i) x - 1.25i has the root x = 0.5 + 0.25i (all exact in binary)
    coef = np.zeros((2, 2, 4))
    coef[0, :, 0] = (1.0, 2.0)
    coef[1, :, 0] = (0.0, -1.25)
    s = System(N=1, n=1, poly_ptr=np.array([0, 2], np.int64), mono_ptr=np.array([0, 1, 1], np.int64),
               var=np.array([0], np.int32), exp=np.array([1], np.uint8), coef=coef,
               xstar=np.array([[0.5, 0.25]]), x0=np.array([[0.5, 0.25]]))
    x = s.point("xstar", L)
    grad, lam = oracle.adjoint(s, x, 2.0 * x, L)
    # -2|x|^2 / conj(c1) = -0.125 (1 + 2i); -2x / conj(c1) = -0.5i
    want = [(-0.125, -0.25), (0.0, -0.5)]
    for t in range(2):
        assert cdiff(cfr(grad[t]), tuple(map(Fraction, want[t]))) <= 16 * ORACLE_OP_BOUND[L]
    assert cdiff(cfr(lam[0]), (Fraction(0), Fraction(1, 2))) <= 16 * ORACLE_OP_BOUND[L]
