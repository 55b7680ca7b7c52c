"""Pins of the oracle's least-squares solver (Section 3).

Modified Gram-Schmidt on [A b] must give Q^H Q = I, A = Q R with R upper
triangular and a real positive diagonal, y = Q^H b (eq. 2), and
||b - A x||^2 = ||R x - y||^2 + z^2.  The solution of R x = y is checked
against numpy.linalg.lstsq in double and against the exact solution of the
normal equations in double double and quad double.
"""

from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_1402_2626_gb300.inputs import cascade_from_fraction
from tests._util import ORACLE_OP_BOUND, cdiff, cfr

LS = (1, 2, 4)


def _rand_matrix(rng, m, n, L):
    A = np.zeros((m, n, 2, L))
    A[..., 0, 0] = rng.standard_normal((m, n))
    A[..., 1, 0] = rng.standard_normal((m, n))
    if L > 1:
        A[..., :, 1] = A[..., :, 0] * 2.0 ** -55 * rng.standard_normal((m, n, 2))
    return A


def _cexact(A):
    return [[cfr(A[i, j]) for j in range(A.shape[1])] for i in range(A.shape[0])]


@pytest.mark.parametrize("L", LS)
def test_mgs_identities_exact(L):
    rng = np.random.default_rng(40 + L)
    m, ncols = 7, 5
    A = _rand_matrix(rng, m, ncols, L)
    Q, R = oracle.mgs(A, L)
    n = ncols - 1
    Ae, Qe, Re = _cexact(A), _cexact(Q), _cexact(R)
    tol = ORACLE_OP_BOUND[L] * 2000
    # R upper triangular, real positive diagonal
    for k in range(ncols):
        for j in range(k):
            assert Re[k][j] == exact.ZERO
        assert Re[k][k][1] == 0 and Re[k][k][0] > 0
    # Q^H Q = I on the first n columns
    for a in range(n):
        for b in range(n):
            s = exact.ZERO
            for i in range(m):
                s = exact.add(s, exact.mul(exact.conj(Qe[i][a]), Qe[i][b]))
            want = exact.ONE if a == b else exact.ZERO
            assert cdiff(s, want) <= tol, (a, b)
    # A = Q R on the first n columns
    for i in range(m):
        for j in range(n):
            s = exact.ZERO
            for k in range(j + 1):
                s = exact.add(s, exact.mul(Qe[i][k], Re[k][j]))
            assert cdiff(s, Ae[i][j]) <= tol * 10
    # y = Q^H b and z^2 = ||b||^2 - ||y||^2 (eq. 2)
    ysq = Fraction(0)
    for k in range(n):
        s = exact.ZERO
        for i in range(m):
            s = exact.add(s, exact.mul(exact.conj(Qe[i][k]), Ae[i][n]))
        assert cdiff(s, Re[k][n]) <= tol * 10
        ysq += Re[k][n][0] ** 2 + Re[k][n][1] ** 2
    bsq = sum(Ae[i][n][0] ** 2 + Ae[i][n][1] ** 2 for i in range(m))
    z = Re[n][n][0]
    assert abs(float(bsq - ysq - z * z)) <= tol * 10 * float(bsq)


def test_lstsq_double_vs_numpy():
    rng = np.random.default_rng(7)
    for m, n in ((12, 8), (8, 8), (30, 3), (5, 1)):
        A = _rand_matrix(rng, m, n + 1, 1)
        _, R = oracle.mgs(A, 1)
        x = oracle.to_complex(oracle.backsub(R, 1))
        Ac = A[:, :n, 0, 0] + 1j * A[:, :n, 1, 0]
        b = A[:, n, 0, 0] + 1j * A[:, n, 1, 0]
        xr, res, *_ = np.linalg.lstsq(Ac, b, rcond=None)
        assert np.allclose(x, xr, rtol=0, atol=1e-12 * np.abs(xr).max())
        # z = ||b - A x|| (eq. 2)
        z = R[n, n, 0, 0]
        assert abs(z - np.linalg.norm(b - Ac @ xr)) <= 1e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("L", [2, 4])
def test_lstsq_vs_exact_normal_equations(L):
    rng = np.random.default_rng(70 + L)
    m, n = 6, 4
    A = _rand_matrix(rng, m, n + 1, L)
    _, R = oracle.mgs(A, L)
    x = oracle.backsub(R, L)
    Ae = _cexact(A)
    G = [[exact.ZERO] * n for _ in range(n)]
    g = [exact.ZERO] * n
    for a in range(n):
        for b in range(n):
            s = exact.ZERO
            for i in range(m):
                s = exact.add(s, exact.mul(exact.conj(Ae[i][a]), Ae[i][b]))
            G[a][b] = s
        s = exact.ZERO
        for i in range(m):
            s = exact.add(s, exact.mul(exact.conj(Ae[i][a]), Ae[i][n]))
        g[a] = s
    xe = exact.solve(G, g)
    scale = max(abs(exact.to_float(v)) for v in xe)
    for k in range(n):
        # cond(A) is O(10) for these shapes
        assert cdiff(cfr(x[k]), xe[k]) <= ORACLE_OP_BOUND[L] * 1e5 * scale


@pytest.mark.parametrize("L", LS)
def test_rank_deficiency_detected(L):
    rng = np.random.default_rng(3)
    A = _rand_matrix(rng, 6, 4, L)
    A[:, 1] = 0.0  # a variable that appears nowhere
    with pytest.raises(oracle.OracleError) as e:
        oracle.mgs(A, L)
    assert e.value.status == oracle.ESINGULAR
    A = _rand_matrix(rng, 6, 4, L)
    A[:, 2] = A[:, 0]  # two equal columns
    with pytest.raises(oracle.OracleError):
        oracle.mgs(A, L)


@pytest.mark.parametrize("L", LS)
def test_consistent_system_has_zero_z(L):
    """b in the range of A gives z = 0 up to rounding and x exactly the combination."""
    rng = np.random.default_rng(11)
    m, n = 8, 3
    A = _rand_matrix(rng, m, n + 1, 1)
    Ac = A[:, :n, 0, 0] + 1j * A[:, :n, 1, 0]
    xt = np.array([1.0, -2.0, 0.5j])
    b = Ac @ xt  # rounded to double: consistent only to ~1e-16
    AL = np.zeros((m, n + 1, 2, L))
    AL[:, :n, :, 0] = A[:, :n, :, 0]
    AL[:, n, 0, 0] = b.real
    AL[:, n, 1, 0] = b.imag
    _, R = oracle.mgs(AL, L)
    assert R[n, n, 0, 0] <= 1e-14 * np.linalg.norm(b)
    x = oracle.to_complex(oracle.backsub(R, L))
    assert np.allclose(x, xt, atol=1e-13)
