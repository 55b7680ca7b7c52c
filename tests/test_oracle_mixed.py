"""Pins of the oracle's mixed-precision Gauss-Newton (double factorisation,
residuals at precision L).

* The result is the generator's exact root x* (a power-of-i point built into
  the system, exact up to the rounding of the constant terms) to the
  precision of L: the refinement reaches the precision of its residuals, not
  the precision of its factorisation.
* With no refinement steps it is plain Gauss-Newton in double (Section 4).
* The refinement converges linearly, each step shrinking the error by at
  least 1e8 (the contraction is about the condition number times the unit
  roundoff of double, 1e-16 kappa).
"""

import numpy as np
import pytest

import oracle
from paper_1402_2626_gb300 import inputs
from tests._util import PARITY_TOL, limb_diff

CASES = [
    ("overdetermined", dict(N=48, n=32, M=(8, 16), k=(1, 6), dmax=4, seed=601)),
    ("square", dict(N=24, n=24, M=(8, 24), k=(1, 5), dmax=3, seed=602)),
]


def _sys(kw):
    return inputs.random_system(kw["N"], kw["n"], kw["M"], kw["k"], kw["dmax"], seed=kw["seed"])


def _err(s, x):
    d = np.array(x, dtype=np.float64, copy=True)
    d[:, :, 0] -= s.xstar
    return float(limb_diff(d, np.zeros_like(d)).max())


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
def test_reaches_exact_root(name, kw, L):
    s = _sys(kw)
    x, hist = oracle.newton_mixed(s, s.point("x0", L), L, 3, 6 if L == 4 else 3)
    assert _err(s, x) <= PARITY_TOL[L]
    # the double phase alone stops near double precision
    xd, _ = oracle.newton_mixed(s, s.point("x0", L), L, 3, 0)
    assert _err(s, xd) > 1e-20


@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
def test_no_refinement_is_double_newton(name, kw):
    s = _sys(kw)
    x, hist = oracle.newton_mixed(s, s.point("x0", 4), 4, 3, 0)
    xd, hd = oracle.newton(s, s.point("x0", 1), 1, 3)
    assert np.array_equal(x[:, :, 0], xd[:, :, 0]) and not np.any(x[:, :, 1:])
    assert hist == hd


def test_linear_contraction_qd():
    s = _sys(CASES[0][1])
    errs = []
    for r in range(0, 6):
        x, _ = oracle.newton_mixed(s, s.point("x0", 4), 4, 3, r)
        errs.append(_err(s, x))
    for a, b in zip(errs, errs[1:]):
        if a > 1e-60:
            assert b <= 1e-8 * a, errs
    assert errs[-1] <= PARITY_TOL[4]
