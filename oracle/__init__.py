"""CPU oracle for the Gauss-Newton hot path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it,
and it shares no code with the CUDA path: the arithmetic lives in
``oracle/oracle.c`` (its own multiword arithmetic built on exact expansions)
and in ``oracle/exact.py`` (exact rationals for tiny inputs).

Complex numbers at precision L (1 = double, 2 = double double, 4 = quad
double) are numpy arrays whose last two axes are ``[2, L]``: real limbs then
imaginary limbs.

Parity unpinned: none.  Every function here is pinned by the tests in
``tests/test_oracle_*.py`` against exact rationals, closed forms, library
routines or invariants.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ESINGULAR = 0, 1, 4

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile oracle/oracle.c into oracle/liboracle.so (gcc, a second or two)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB_OVERRIDE lets the mutation tests load a deliberately
            # broken copy of the oracle in a child process.
            path = os.environ.get("ORACLE_LIB_OVERRIDE") or build()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            i64p = C.POINTER(C.c_int64)
            L.o_real_op.argtypes = [C.c_int, C.c_int, dp, dp, dp]
            L.o_cplx_op.argtypes = [C.c_int, C.c_int, dp, dp, dp]
            L.o_eval.argtypes = [
                C.c_int, C.c_int, C.c_int32, C.c_int32, i64p, i64p,
                C.POINTER(C.c_int32), C.POINTER(C.c_uint8), dp, C.c_int, dp,
                C.c_int32, C.c_int32, dp, dp, C.c_int64, C.c_int, i64p,
            ]
            L.o_speelpenning.argtypes = [C.c_int, C.c_int, dp, dp, dp]
            L.o_speelpenning.restype = C.c_int64
            L.o_mgs.argtypes = [C.c_int, C.c_int32, C.c_int32, dp, C.c_int64, dp, C.c_int32, C.c_int]
            L.o_backsub.argtypes = [C.c_int, C.c_int32, dp, C.c_int32, dp]
            L.o_axpy_update.argtypes = [C.c_int, C.c_int32, dp, dp]
            L.o_adjoint.argtypes = [C.c_int, C.c_int32, C.c_int32, dp, C.c_int64, dp, C.c_int32,
                                    dp, dp, dp]
            L.o_monomials.argtypes = [C.c_int, C.c_int64, i64p, C.POINTER(C.c_int32),
                                      C.POINTER(C.c_uint8), dp, dp]
            L.o_coef_grad.argtypes = [C.c_int, C.c_int32, i64p, dp, dp, dp]
            _lib = L
    return _lib


def _p(a, ct=C.c_double):
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"oracle {what} failed with status {status}")
        self.status = status


# -- primitives ---------------------------------------------------------------

REAL_OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3, "sqrt": 4}
CPLX_OPS = {"add": 0, "sub": 1, "mul": 2, "conj_mul": 3, "abs2": 4, "div_real": 5}


def real_op(L: int, op: str, a, b=None) -> np.ndarray:
    a = _f64(a).reshape(L)
    b = _f64(a if b is None else b).reshape(L)
    c = np.zeros(L)
    st = lib().o_real_op(L, REAL_OPS[op], _p(a), _p(b), _p(c))
    if st:
        raise OracleError(st, op)
    return c


def cplx_op(L: int, op: str, a, b=None) -> np.ndarray:
    a = _f64(a).reshape(2, L)
    b = _f64(a if b is None else b).reshape(2, L)
    c = np.zeros((2, L))
    st = lib().o_cplx_op(L, CPLX_OPS[op], _p(a), _p(b), _p(c))
    if st:
        raise OracleError(st, op)
    return c


def speelpenning(L: int, xs):
    """Value and gradient of x_1 * ... * x_k; returns (value, grad, nmul)."""
    xs = _f64(xs).reshape(-1, 2, L)
    k = xs.shape[0]
    val = np.zeros((2, L))
    grad = np.zeros((max(k, 1), 2, L))
    nmul = lib().o_speelpenning(L, k, _p(xs), _p(val), _p(grad))
    return val, grad[:k], int(nmul)


# -- evaluation and differentiation ---------------------------------------------


def evaluate(system, x, L: int, mode: str = "reverse", rows=None, jacobian=True,
             nthreads: int = 1):
    """f and J of ``system`` at ``x`` ([n, 2, >=L]) in precision L.

    Returns ``(f [nr, 2, L], J [nr, n, 2, L] or None, nmul)`` for the rows
    ``rows = (row0, row1)`` (default all).  ``mode`` is "definition" or
    "reverse".
    """
    n, N = system.n, system.N
    r0, r1 = (0, N) if rows is None else rows
    nr = r1 - r0
    x = _f64(np.asarray(x)[..., :L]).reshape(n, 2, L)
    coef = system.coef_limbs(L)
    f = np.zeros((nr, 2, L))
    Jcm = np.zeros((n, max(nr, 1), 2, L)) if jacobian else None
    nmul = np.zeros(1, dtype=np.int64)
    st = lib().o_eval(
        L, 0 if mode == "definition" else 1, N, n,
        _p(system.poly_ptr, C.c_int64), _p(system.mono_ptr, C.c_int64),
        _p(system.var, C.c_int32), _p(system.exp, C.c_uint8),
        _p(coef), L, _p(x), r0, r1, _p(f),
        _p(Jcm) if jacobian else None, max(nr, 1), nthreads, _p(nmul, C.c_int64),
    )
    if st:
        raise OracleError(st, "eval")
    J = None
    if jacobian:
        J = np.ascontiguousarray(Jcm[:, :nr].transpose(1, 0, 2, 3))
    return f, J, int(nmul[0])


# -- least squares --------------------------------------------------------------


def mgs(A, L: int, nthreads: int = 1):
    """MGS on the augmented matrix A = [J, b] given as [m, ncols, 2, L].

    Returns (Q-overwritten A [m, ncols, 2, L], R [ncols, ncols, 2, L]); raises
    OracleError(ESINGULAR) on a rank-deficient leading block.
    """
    A = _f64(A)
    m, ncols = A.shape[0], A.shape[1]
    Acm = np.array(A.transpose(1, 0, 2, 3), order="C", copy=True)  # never alias the input
    Rcm = np.zeros((ncols, ncols, 2, L))
    st = lib().o_mgs(L, m, ncols, _p(Acm), m, _p(Rcm), ncols, nthreads)
    if st:
        raise OracleError(st, "mgs")
    return (np.ascontiguousarray(Acm.transpose(1, 0, 2, 3)),
            np.ascontiguousarray(Rcm.transpose(1, 0, 2, 3)))


def backsub(R, L: int):
    """Solve R[:n,:n] x = R[:n, n] for the (n+1) x (n+1) factor of [A b]."""
    R = _f64(R)
    ncols = R.shape[0]
    n = ncols - 1
    Rcm = np.array(R.transpose(1, 0, 2, 3), order="C", copy=True)
    x = np.zeros((max(n, 1), 2, L))
    st = lib().o_backsub(L, n, _p(Rcm), ncols, _p(x))
    if st:
        raise OracleError(st, "backsub")
    return x[:n]


def add_vec(x, dx, L: int):
    x = _f64(x).copy()
    dx = _f64(dx)
    lib().o_axpy_update(L, x.shape[0], _p(x), _p(dx))
    return x


def augmented(f, J):
    """[J, -f] as [m, n+1, 2, L] (Section 4: A = J_f(x0), b = -f(x0))."""
    return np.concatenate([J, -f[:, None]], axis=1)


def newton_step(system, x, L: int, nthreads: int = 1):
    """One Gauss-Newton step (Section 4); returns (x1, dx, f, R)."""
    f, J, _ = evaluate(system, x, L, "reverse", nthreads=nthreads)
    _, R = mgs(augmented(f, J), L, nthreads=nthreads)
    dx = backsub(R, L)
    return add_vec(x, dx, L), dx, f, R


def newton(system, x0, L: int, steps: int, nthreads: int = 1):
    """``steps`` Gauss-Newton steps; returns (x, [(|f|_2, |dx|_2) per step])."""
    x = _f64(np.asarray(x0)[..., :L]).reshape(system.n, 2, L).copy()
    hist = []
    for _ in range(steps):
        x, dx, f, _ = newton_step(system, x, L, nthreads=nthreads)
        hist.append((float(np.sqrt((f[:, :, 0] ** 2).sum())),
                     float(np.sqrt((dx[:, :, 0] ** 2).sum()))))
    return x, hist


# -- mixed precision: double factorisation, residuals at precision L --------------


def newton_mixed(system, x0, L: int, d_steps: int, refine_steps: int, nthreads: int = 1):
    """Gauss-Newton in two phases (an extension past the paper; Section 5.2
    notes that the linear solve dominates a Newton step and that iterative
    methods in double arithmetic may do well):

    1. ``d_steps`` full Gauss-Newton steps (Section 4) in double precision from
       the leading limbs of x0, keeping the factors Q, R of the last step's
       [J, -f] (Section 3);
    2. ``refine_steps`` refinement steps at precision L with those factors
       frozen: b = -f(x) evaluated at precision L (Section 2) and rounded to
       double, y = Q^H b in double (terms summed in row order), R dx = y by
       back substitution in double, x <- x + dx at precision L.

    Returns (x [n, 2, L], [(|f|_2, |dx|_2) per step]).
    """
    n = system.n
    x = np.zeros((n, 2, 1))
    x[:, :, 0] = np.asarray(x0)[:, :, 0]
    hist = []
    Q = R = None
    for _ in range(d_steps):
        f, J, _ = evaluate(system, x, 1, "reverse", nthreads=nthreads)
        Q, R = mgs(augmented(f, J), 1, nthreads=nthreads)
        dx = backsub(R, 1)
        x = add_vec(x, dx, 1)
        hist.append((float(np.sqrt((f[:, :, 0] ** 2).sum())), float(np.sqrt((dx[:, :, 0] ** 2).sum()))))
    xl = np.zeros((n, 2, L))
    xl[:, :, 0] = x[:, :, 0]
    for _ in range(refine_steps):
        f, _, _ = evaluate(system, xl, L, "reverse", jacobian=False, nthreads=nthreads)
        b = -f[:, :, :1]
        Ry = R.copy()
        for k in range(n):
            acc = np.zeros((2, 1))
            for i in range(system.N):
                acc = cplx_op(1, "add", acc, cplx_op(1, "conj_mul", Q[i, k], b[i]))
            Ry[k, n] = acc
        dx = backsub(Ry, 1)
        dxl = np.zeros((n, 2, L))
        dxl[:, :, 0] = dx[:, :, 0]
        xl = add_vec(xl, dxl, L)
        hist.append((float(np.sqrt((f[:, :, 0] ** 2).sum())), float(np.sqrt((dx[:, :, 0] ** 2).sum()))))
    return xl, hist


# -- adjoint (gradient with respect to the coefficients) ------------------------


def monomials(system, x, L: int) -> np.ndarray:
    """m_t = x^{a_t} for every term ([T, 2, L]; 1 for a constant term)."""
    x = _f64(np.asarray(x)[..., :L]).reshape(system.n, 2, L)
    out = np.zeros((system.T, 2, L))
    st = lib().o_monomials(L, system.T, _p(system.mono_ptr, C.c_int64), _p(system.var, C.c_int32),
                           _p(system.exp, C.c_uint8), _p(x), _p(out))
    if st:
        raise OracleError(st, "monomials")
    return out


def adjoint(system, x, g, L: int, nthreads: int = 1):
    """Gradient of a real loss with respect to every coefficient at a root x.

    ``g`` ([n, 2, L]) is the loss gradient dL/dRe x + i dL/dIm x at x.  The
    root moves by dx = -J^+ (df/dc) dc (implicit function theorem at the
    Gauss-Newton fixed point of Section 4, J = QR as in Section 3), so the
    coefficient gradient is grad_t = -lambda_{i(t)} conj(x^{a_t}) with
    lambda = Q R^{-H} g.  Every coefficient, the constant terms included,
    counts as an independent input.  Returns (grad [T, 2, L], lambda [N, 2, L]).
    """
    n, N = system.n, system.N
    x = _f64(np.asarray(x)[..., :L]).reshape(n, 2, L)
    g = _f64(np.asarray(g)[..., :L]).reshape(n, 2, L)
    f, J, _ = evaluate(system, x, L, "reverse", nthreads=nthreads)
    Q, R = mgs(augmented(f, J), L, nthreads=nthreads)  # leading n columns: J = QR
    Qcm = np.ascontiguousarray(Q[:, :n].transpose(1, 0, 2, 3))
    Rcm = np.ascontiguousarray(R[:n, :n].transpose(1, 0, 2, 3))
    w = np.zeros((max(n, 1), 2, L))
    lam = np.zeros((max(N, 1), 2, L))
    st = lib().o_adjoint(L, N, n, _p(Qcm), N, _p(Rcm), n, _p(g), _p(w), _p(lam))
    if st:
        raise OracleError(st, "adjoint")
    lam = lam[:N]
    mono = monomials(system, x, L)
    grad = np.zeros((system.T, 2, L))
    lib().o_coef_grad(L, N, _p(system.poly_ptr, C.c_int64), _p(lam), _p(mono), _p(grad))
    return grad, lam


def to_complex(a) -> np.ndarray:
    """Leading limb as numpy complex (for double-precision comparisons)."""
    a = np.asarray(a)
    return a[..., 0, 0] + 1j * a[..., 1, 0]
