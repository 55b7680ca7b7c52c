"""Pins of the oracle's evaluation and differentiation (Section 2).

* Speelpenning: the gradient of x_1 ... x_k is the vector of products of all
  the other variables (Section 2.2), checked exactly, and the reverse mode
  uses 3k-5 multiplications, the straightforward way k^2-k-1
  (tests/golden/operation_counts.txt).
* f and J of whole systems against the exact-rational definition
  (oracle/exact.py), in both oracle modes and all three precisions.
* J against central differences of f in quad double.
* f vanishes at the root built into the generated systems, whose constant
  terms come from an independent exact Gaussian-integer computation.
"""

import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_1402_2626_gb300 import inputs
from tests._util import ORACLE_OP_BOUND, cdiff, cfr, limb_diff, term_scales

HERE = os.path.dirname(os.path.abspath(__file__))
LS = (1, 2, 4)


def _golden_counts():
    rows = []
    with open(os.path.join(HERE, "golden", "operation_counts.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                kind, k, m = line.split()
                rows.append((kind, int(k), int(m)))
    return rows


def _rand_points(rng, k, L):
    th = 2 * np.pi * rng.random(k)
    r = 0.5 + rng.random(k)
    x = np.zeros((k, 2, L))
    x[:, 0, 0] = r * np.cos(th)
    x[:, 1, 0] = r * np.sin(th)
    if L > 1:  # nonzero lower limbs so every limb takes part
        x[:, 0, 1] = x[:, 0, 0] * 2.0 ** -60 * rng.standard_normal(k)
        x[:, 1, 1] = x[:, 1, 0] * 2.0 ** -60 * rng.standard_normal(k)
    return x


@pytest.mark.parametrize("kind,k,m", _golden_counts())
def test_operation_counts(kind, k, m):
    rng = np.random.default_rng(k)
    if kind == "speelpenning":
        _, _, nmul = oracle.speelpenning(1, _rand_points(rng, k, 1))
        assert nmul == m == 3 * k - 5
    else:
        if k > 16:
            pytest.skip("straightforward mode is quadratic")
        # one monomial x_1 ... x_k with coefficient 1 in a 1-polynomial system
        s = inputs.System(
            N=1, n=k, poly_ptr=np.array([0, 1], np.int64), mono_ptr=np.array([0, k], np.int64),
            var=np.arange(k, dtype=np.int32), exp=np.ones(k, np.uint8),
            coef=np.array([[[1.0, 0, 0, 0], [0, 0, 0, 0]]]))
        _, _, nmul = oracle.evaluate(s, _rand_points(rng, k, 1), 1, "definition")
        assert nmul == m == k * k - k - 1


@pytest.mark.parametrize("L", LS)
@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 5, 8, 9, 16, 31, 32, 33])
def test_speelpenning_closed_form(L, k):
    rng = np.random.default_rng(1000 * L + k)
    xs = _rand_points(rng, k, L)
    val, grad, nmul = oracle.speelpenning(L, xs)
    ex = [cfr(x) for x in xs]
    prod = exact.ONE
    for e in ex:
        prod = exact.mul(prod, e)
    bound = ORACLE_OP_BOUND[L] * 4 * max(k, 1)
    assert cdiff(cfr(val), prod) <= bound * abs(exact.to_float(prod))
    for s in range(k):
        other = exact.ONE
        for r, e in enumerate(ex):
            if r != s:
                other = exact.mul(other, e)
        assert cdiff(cfr(grad[s]), other) <= bound * abs(exact.to_float(other)), (s, k)
    assert nmul == (3 * k - 5 if k >= 2 else 0)


def _small_systems():
    out = []
    for seed in range(4):
        out.append(inputs.random_system(4, 4, (1, 5), (1, 4), 5, seed=10 + seed, exact_root=True))
    out.append(inputs.random_system(3, 5, 6, 5, 2, seed=77, exact_root=False))
    out.append(inputs.random_system(5, 3, (2, 4), (1, 3), 4, seed=78, constant=False))
    return out


@pytest.mark.parametrize("L", LS)
@pytest.mark.parametrize("mode", ["reverse", "definition"])
def test_eval_vs_exact(L, mode):
    for s in _small_systems():
        rng = np.random.default_rng(5)
        x = _rand_points(rng, s.n, L)
        f, J, _ = oracle.evaluate(s, x, L, mode)
        fe, Je = exact.evaluate(s, x, L=L)
        Sf, SJ = term_scales(s, x)
        nterm = max(int(np.diff(s.poly_ptr).max()), 1)
        kmax = max(int(np.diff(s.mono_ptr).max()), 1)
        bound = ORACLE_OP_BOUND[L] * 8 * (nterm + 3 * kmax + 10)
        for i in range(s.N):
            assert cdiff(cfr(f[i]), fe[i]) <= bound * Sf[i], (i, mode)
            for v in range(s.n):
                want = Je.get((i, v), exact.ZERO)
                if want == exact.ZERO and SJ[i, v] == 0:
                    assert not np.any(J[i, v]), "entry with no term must be exactly 0"
                else:
                    assert cdiff(cfr(J[i, v]), want) <= bound * SJ[i, v], (i, v, mode)


@pytest.mark.parametrize("L", [2, 4])
def test_reverse_matches_definition_medium(L):
    s = inputs.random_system(12, 16, (10, 20), (1, 12), 4, seed=99)
    x = s.point("x0", L)
    f1, J1, n1 = oracle.evaluate(s, x, L, "reverse")
    f2, J2, n2 = oracle.evaluate(s, x, L, "definition")
    Sf, SJ = term_scales(s, x)
    tol = ORACLE_OP_BOUND[L] * 2000
    assert np.all(limb_diff(f1, f2) <= tol * Sf)
    assert np.all(limb_diff(J1, J2) <= tol * SJ + 0.0)
    assert n1 < n2  # reverse mode shares work


def test_jacobian_central_differences_qd():
    """J[:, v] ~ (f(x + h e_v) - f(x - h e_v)) / 2h, f holomorphic, QD, h = 2^-70."""
    s = inputs.random_system(6, 5, (3, 6), (1, 4), 4, seed=123)
    L = 4
    x = s.point("x0", L)
    f, J, _ = oracle.evaluate(s, x, L)
    h = 2.0 ** -70
    _, SJ = term_scales(s, x)
    for v in range(s.n):
        xp = x.copy()
        xm = x.copy()
        hv = np.array([h, 0, 0, 0])
        xp[v, 0] = oracle.real_op(4, "add", x[v, 0], hv)
        xm[v, 0] = oracle.real_op(4, "sub", x[v, 0], hv)
        fp, _, _ = oracle.evaluate(s, xp, L, jacobian=False)
        fm, _, _ = oracle.evaluate(s, xm, L, jacobian=False)
        for i in range(s.N):
            d = exact.sub(cfr(fp[i]), cfr(fm[i]))
            fd = (d[0] / Fraction(2 * h), d[1] / Fraction(2 * h))
            # truncation ~ h^2, rounding ~ 2^-212 / h: both below 1e-40
            assert cdiff(cfr(J[i, v]), fd) <= 1e-38 * max(SJ[i, v], 1.0), (i, v)


@pytest.mark.parametrize("L", LS)
def test_generated_root_is_root(L):
    """f(x*) vanishes up to the rounding of the constant terms (gn32 workload)."""
    s = inputs.workload("gn32")
    f, _, _ = oracle.evaluate(s, s.point("xstar", L), L, jacobian=False)
    Sf, _ = term_scales(s, s.point("xstar", L))
    assert np.all(limb_diff(f, np.zeros_like(f)) <= ORACLE_OP_BOUND[L] * 8 * (s.T // s.N + 40) * Sf)
    # and it does not vanish at the perturbed start point
    f0, _, _ = oracle.evaluate(s, s.point("x0", L), L, jacobian=False)
    assert np.abs(f0[:, :, 0]).max() > 1e-8


def test_generated_root_exact_mode():
    """Exact f(x*) equals minus the rounding error of each stored constant term."""
    s = inputs.random_system(3, 4, 5, (2, 4), 3, seed=31)
    fe, _ = exact.evaluate(s, s.point("xstar", 1), L=4)
    for i in range(s.N):
        # rounding of the 4-limb constant: below 2^-200 relative to the term scale
        assert abs(exact.to_float(fe[i])) <= 2.0 ** -200 * 10


def test_rejects_bad_support():
    s = inputs.random_system(2, 3, 2, 2, 2, seed=1)
    bad = inputs.System(N=s.N, n=s.n, poly_ptr=s.poly_ptr, mono_ptr=s.mono_ptr,
                        var=s.var.copy(), exp=s.exp.copy(), coef=s.coef)
    bad.var[0] = 7
    with pytest.raises(oracle.OracleError):
        oracle.evaluate(bad, s.point("x0", 1), 1)
    bad.var[0] = s.var[0]
    bad.exp[0] = 0
    with pytest.raises(oracle.OracleError):
        oracle.evaluate(bad, s.point("x0", 1), 1)
