"""Seeded synthetic polynomial systems in sparse distributed form.

This module only builds inputs. Both the CUDA path and the CPU oracle read
them; it contains none of the method's evaluation, differentiation or
least-squares arithmetic.

A system is stored the way the Problem Statement of the paper (Section 1)
describes it: fully expanded, keeping only monomials with a nonzero
coefficient.  Monomial ``t`` of polynomial ``i`` lives in
``[poly_ptr[i], poly_ptr[i+1])``; its support is
``var[mono_ptr[t]:mono_ptr[t+1]]`` with exponents ``exp[...]`` (all >= 1,
Section 2.1, eq. 1).  A monomial with an empty support is a constant term.

Coefficients are stored as a cascade of 4 doubles per real part
(``coef[t, 0, :]`` real limbs, ``coef[t, 1, :]`` imaginary limbs).  Limb
``l+1`` is the nearest double to what limbs ``0..l`` leave over, so the
first ``L`` limbs are the nearest ``L``-limb cascade for every ``L`` in
{1, 2, 4}.  Only the constant terms use more than one limb.

Recipe of the random workloads (the paper's own benchmarks are closed-form
systems; these stand in for them):

* each polynomial has ``M`` non-constant monomials plus one constant term;
* a monomial's support is a uniform ``k``-subset of the ``n`` variables
  without replacement, stored sorted ascending; exponents are i.i.d. uniform
  in ``{1..dmax}``; monomials inside one polynomial are distinct
  (rejection sampling);
* coefficients and the root ``x*`` are unit-modulus, ``(cos 2 pi u, sin 2 pi u)``
  rounded to double;
* the constant term of polynomial ``i`` is ``-sum_t c_t x*^{a_t}``, computed
  exactly in Gaussian-integer arithmetic on the double inputs and then
  rounded to the 4-limb cascade, so ``x*`` is a root of the stored system up
  to one rounding of the constant term;
* the start point is ``x0_j = x*_j + 1e-6 exp(i phi_j)`` rounded to double.

Random streams come from numpy's PCG64 through ``SeedSequence.spawn``: one
stream each for supports, exponents, coefficients, the root and the
perturbation.
"""

from __future__ import annotations

import functools
import math
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

BASE_SEED = 0x14022626

__all__ = [
    "cyclic",
    "cyclic_homotopy",
    "chandrasekhar",
    "Batch",
    "random_batch",
    "batch_workload",
    "System",
    "random_system",
    "workload",
    "WORKLOADS",
    "limbs_of",
    "cascade_from_fraction",
]


@dataclass
class System:
    """A polynomial system in sparse distributed form (host arrays)."""

    N: int
    n: int
    poly_ptr: np.ndarray  # int64 [N+1]
    mono_ptr: np.ndarray  # int64 [T+1]
    var: np.ndarray  # int32 [nnz]
    exp: np.ndarray  # uint8 [nnz]
    coef: np.ndarray  # float64 [T, 2, 4]
    xstar: np.ndarray | None = None  # float64 [n, 2]
    x0: np.ndarray | None = None  # float64 [n, 2]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def T(self) -> int:
        return int(self.mono_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.var.shape[0])

    def coef_limbs(self, L: int) -> np.ndarray:
        """Coefficients with the first L limbs per part, [T, 2, L] contiguous."""
        return np.ascontiguousarray(self.coef[:, :, :L])

    def point(self, which: str, L: int) -> np.ndarray:
        """x* or x0 as [n, 2, L] (higher limbs zero)."""
        src = self.xstar if which == "xstar" else self.x0
        out = np.zeros((self.n, 2, L), dtype=np.float64)
        out[:, :, 0] = src
        return out


def limbs_of(value: Fraction, L: int) -> list[float]:
    """Nearest-double cascade of an exact rational with L limbs."""
    return cascade_from_fraction(value, L)


def cascade_from_fraction(value: Fraction, L: int) -> list[float]:
    out = []
    rem = Fraction(value)
    for _ in range(L):
        d = float(rem)  # correctly rounded (round half to even)
        out.append(d)
        rem -= Fraction(d)
    return out


# -- exact Gaussian-integer values (A + iB) * 2**E ----------------------------


def _exact(re: float, im: float):
    a, b = re.as_integer_ratio()
    c, d = im.as_integer_ratio()
    ea = -(b.bit_length() - 1)
    ec = -(d.bit_length() - 1)
    E = min(ea, ec)
    return (a << (ea - E), c << (ec - E), E)


def _gmul(x, y):
    a1, b1, e1 = x
    a2, b2, e2 = y
    return (a1 * a2 - b1 * b2, a1 * b2 + b1 * a2, e1 + e2)


def _gsum(terms):
    if not terms:
        return (0, 0, 0)
    E = min(t[2] for t in terms)
    A = 0
    B = 0
    for a, b, e in terms:
        A += a << (e - E)
        B += b << (e - E)
    return (A, B, E)


def _to_fraction(a: int, e: int) -> Fraction:
    return Fraction(a) * (Fraction(2) ** e)


def _unit(rng, size):
    th = 2.0 * math.pi * rng.random(size)
    return np.stack([np.cos(th), np.sin(th)], axis=-1)


def random_system(
    N: int,
    n: int,
    M,
    k,
    dmax: int,
    seed: int,
    constant: bool = True,
    exact_root: bool = True,
    dmin: int = 1,
    name: str = "",
) -> System:
    """Random system with an exact root built in.

    ``M`` and ``k`` are ints or ``(lo, hi)`` inclusive ranges drawn per
    polynomial (``M``) and per monomial (``k``).
    """
    ss = np.random.SeedSequence(seed)
    r_sup, r_exp, r_coef, r_root, r_pert = [np.random.default_rng(s) for s in ss.spawn(5)]

    def draw(spec, rng):
        if isinstance(spec, tuple):
            return int(rng.integers(spec[0], spec[1] + 1))
        return int(spec)

    xstar = _unit(r_root, n)
    phi = 2.0 * math.pi * r_pert.random(n)
    x0 = xstar + 1e-6 * np.stack([np.cos(phi), np.sin(phi)], axis=-1)

    poly_ptr = [0]
    mono_ptr = [0]
    var_l = []
    exp_l = []
    coefs = []  # list of (re, im) doubles for non-constant terms; None marks constant
    for i in range(N):
        Mi = draw(M, r_sup)
        seen = set()
        monos = []
        while len(monos) < Mi:
            ki = min(draw(k, r_sup), n)
            vs = np.sort(r_sup.choice(n, size=ki, replace=False)).astype(np.int32)
            ds = r_exp.integers(dmin, dmax + 1, size=ki).astype(np.uint8)
            key = (vs.tobytes(), ds.tobytes())
            if key in seen or ki == 0:
                continue
            seen.add(key)
            monos.append((vs, ds))
        cs = _unit(r_coef, Mi)
        for (vs, ds), c in zip(monos, cs):
            var_l.append(vs)
            exp_l.append(ds)
            mono_ptr.append(mono_ptr[-1] + len(vs))
            coefs.append((float(c[0]), float(c[1])))
        if constant:
            mono_ptr.append(mono_ptr[-1])
            coefs.append(None)
        poly_ptr.append(len(mono_ptr) - 1)

    T = len(mono_ptr) - 1
    var = np.concatenate(var_l).astype(np.int32) if var_l else np.zeros(0, np.int32)
    exp = np.concatenate(exp_l).astype(np.uint8) if exp_l else np.zeros(0, np.uint8)
    coef = np.zeros((T, 2, 4), dtype=np.float64)
    for t, c in enumerate(coefs):
        if c is not None:
            coef[t, 0, 0] = c[0]
            coef[t, 1, 0] = c[1]

    sys_ = System(
        N=N,
        n=n,
        poly_ptr=np.asarray(poly_ptr, dtype=np.int64),
        mono_ptr=np.asarray(mono_ptr, dtype=np.int64),
        var=var,
        exp=exp,
        coef=coef,
        xstar=xstar,
        x0=x0,
        name=name,
        meta=dict(N=N, n=n, M=M, k=k, dmax=dmax, seed=seed),
    )
    if constant and exact_root:
        _set_constants(sys_)
    return sys_


def _set_constants(s: System) -> None:
    """Constant term of each polynomial = -sum of its other terms at x*, exactly."""
    dmax = int(s.exp.max()) if s.nnz else 1
    P = []
    for v in range(s.n):
        row = [None, _exact(float(s.xstar[v, 0]), float(s.xstar[v, 1]))]
        for p in range(2, dmax + 1):
            row.append(_gmul(row[p - 1], row[1]))
        P.append(row)
    for i in range(s.N):
        terms = []
        const_t = []
        for t in range(int(s.poly_ptr[i]), int(s.poly_ptr[i + 1])):
            a, b = int(s.mono_ptr[t]), int(s.mono_ptr[t + 1])
            if a == b:
                const_t.append(t)
                continue
            acc = _exact(float(s.coef[t, 0, 0]), float(s.coef[t, 1, 0]))
            for v, d in zip(s.var[a:b], s.exp[a:b]):
                acc = _gmul(acc, P[int(v)][int(d)])
            terms.append(acc)
        A, B, E = _gsum(terms)
        re = -_to_fraction(A, E)
        im = -_to_fraction(B, E)
        for t in const_t[:1]:
            s.coef[t, 0, :] = cascade_from_fraction(re, 4)
            s.coef[t, 1, :] = cascade_from_fraction(im, 4)


# -- the paper's closed-form benchmark systems ------------------------------------


def _cyclic_windows(n: int, i: int) -> np.ndarray:
    """Supports of polynomial i of cyclic n-roots: the n windows
    {j, ..., j+i-1 mod n}, each sorted ascending ([n, i])."""
    w = (np.arange(n)[:, None] + np.arange(i)[None, :]) % n
    return np.sort(w, axis=1).astype(np.int32)


def cyclic(n: int, seed: int = 0) -> System:
    """The cyclic n-roots system (Section 5.3, eq. 7): for i = 1 .. n-1 the
    sum over j = 0 .. n-1 of the products x_j x_{j+1} ... x_{j+i-1} (indices
    mod n), and x_0 x_1 ... x_{n-1} - 1.  Coefficients 1 (and the constant
    -1); every exponent 1.  ``x0`` is a seeded point of unit-modulus
    coordinates (cos 2 pi u, sin 2 pi u), the kind of point the paper's
    evaluation runs use; there is no built-in root (``xstar`` is None)."""
    supports = [_cyclic_windows(n, i) for i in range(1, n)]
    supports.append(np.arange(n, dtype=np.int32)[None, :])
    poly_ptr = [0]
    lengths = []
    for i, w in enumerate(supports):
        lengths.extend([w.shape[1]] * w.shape[0])
        if i == n - 1:
            lengths.append(0)  # the constant -1
        poly_ptr.append(len(lengths))
    mono_ptr = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=mono_ptr[1:])
    var = np.concatenate([w.ravel() for w in supports]).astype(np.int32)
    T = len(lengths)
    coef = np.zeros((T, 2, 4))
    coef[:, 0, 0] = 1.0
    coef[T - 1, 0, 0] = -1.0
    rng = np.random.default_rng(np.random.SeedSequence(BASE_SEED + 6000 + seed))
    return System(N=n, n=n, poly_ptr=np.asarray(poly_ptr, dtype=np.int64), mono_ptr=mono_ptr,
                  var=var, exp=np.ones(var.shape[0], dtype=np.uint8), coef=coef, xstar=None,
                  x0=_unit(rng, n), name=f"cyclic{n}", meta=dict(n=n, seed=seed))


def cyclic_homotopy(n: int, t: float = 1.0 - 2.0 ** -20, seed: int = 0) -> System:
    """The Newton homotopy of Section 5.3 on cyclic n-roots: f(x) - t f(z) = 0,
    which z solves at t = 1, with ``x0`` = z.  The paper draws z at random in
    C^n; here z_k = i^(e_k) with e_k uniform in {0, 1, 2, 3}, so that every
    product in f(z) is a power of i and f(z) is a Gaussian integer found by
    counting, and t f(z) is exact in double (t = 1 - 2^-20 by default).  Each
    polynomial gets the constant -t f_i(z) (the last one -1 - t f_n(z))."""
    base = cyclic(n, seed)
    rng = np.random.default_rng(np.random.SeedSequence(BASE_SEED + 7000 + seed))
    e = rng.integers(0, 4, size=n)
    pref = np.concatenate([[0], np.cumsum(np.concatenate([e, e]))])  # window sums via prefix sums
    fz = []
    for i in range(1, n):
        pw = (pref[np.arange(n) + i] - pref[np.arange(n)]) % 4
        cnt = np.bincount(pw, minlength=4)
        fz.append((int(cnt[0] - cnt[2]), int(cnt[1] - cnt[3])))
    q = int(e.sum()) % 4
    prod_z = [(1, 0), (0, 1), (-1, 0), (0, -1)][q]
    fz.append((prod_z[0] - 1, prod_z[1]))
    poly_ptr = [0]
    mono_ptr = [0]
    coef_rows = []
    for i in range(n):
        t0, t1 = int(base.poly_ptr[i]), int(base.poly_ptr[i + 1])
        last = i == n - 1
        for tt in range(t0, t1 - (1 if last else 0)):
            mono_ptr.append(int(base.mono_ptr[tt + 1]))
            coef_rows.append((1.0, 0.0))
        # constant: -t f_i(z), and for the last polynomial -1 - t f_n(z)
        c = (-t * fz[i][0] - (1.0 if last else 0.0), -t * fz[i][1])
        mono_ptr.append(mono_ptr[-1])
        coef_rows.append(c)
        poly_ptr.append(len(mono_ptr) - 1)
    T = len(coef_rows)
    coef = np.zeros((T, 2, 4))
    coef[:, 0, 0] = [c[0] for c in coef_rows]
    coef[:, 1, 0] = [c[1] for c in coef_rows]
    z = np.stack([np.real(1j ** e), np.imag(1j ** e)], axis=-1).round()
    return System(N=n, n=n, poly_ptr=np.asarray(poly_ptr, dtype=np.int64),
                  mono_ptr=np.asarray(mono_ptr, dtype=np.int64), var=base.var, exp=base.exp,
                  coef=coef, xstar=None, x0=z, name=f"cyclic{n}-homotopy",
                  meta=dict(n=n, t=t, seed=seed, z_exponents=e))


def _cascade_ratio(p: int, q: int, L: int) -> list[float]:
    """Nearest-double cascade of the rational p/q (q > 0) with L limbs, in
    integer arithmetic (CPython's int / int is correctly rounded)."""
    out = []
    num, den = p, q
    for _ in range(L):
        d = num / den if num else 0.0
        out.append(d)
        a, b = d.as_integer_ratio()  # d = a / b, b a power of two
        num, den = num * b - a * den, den * b
    return out


def chandrasekhar(n: int, c: Fraction = Fraction(33, 64)) -> System:
    """The Chandrasekhar H-equation system (Section 5.2, eq. 6), read with
    j = 1 .. n (the equation prints j = 0 .. n-1 beside the 1-indexed H):
    f_i = 2n H_i - c H_i sum_{j=1..n} (i / (i + j)) H_j - 2n, i = 1 .. n.
    Terms of polynomial i: 2n H_i; -c i/(i+j) H_i H_j for j != i; -c/2 H_i^2;
    the constant -2n.  Coefficients are rational: stored as the nearest
    4-limb cascades.  ``x0`` is H = 1 (the paper's start); no built-in root."""
    cn, cd = c.numerator, c.denominator
    poly_ptr = [0]
    mono_ptr = [0]
    var = []
    exp = []
    coefs = []  # (p, q): the coefficient p / q
    for i in range(1, n + 1):
        # linear term
        var.append(i - 1)
        exp.append(1)
        mono_ptr.append(len(var))
        coefs.append((2 * n, 1))
        for j in range(1, n + 1):
            if j == i:
                var.append(i - 1)
                exp.append(2)
            else:
                a, b = (i - 1, j - 1) if i < j else (j - 1, i - 1)
                var.append(a)
                var.append(b)
                exp.append(1)
                exp.append(1)
            coefs.append((-cn * i, cd * (i + j)))  # j = i: -c i / 2i = -c/2
            mono_ptr.append(len(var))
        mono_ptr.append(len(var))  # constant
        coefs.append((-2 * n, 1))
        poly_ptr.append(len(mono_ptr) - 1)
    T = len(coefs)
    coef = np.zeros((T, 2, 4))
    for t, (pq, qq) in enumerate(coefs):
        coef[t, 0, :] = _cascade_ratio(pq, qq, 4)
    return System(N=n, n=n, poly_ptr=np.asarray(poly_ptr, dtype=np.int64),
                  mono_ptr=np.asarray(mono_ptr, dtype=np.int64), var=np.asarray(var, dtype=np.int32),
                  exp=np.asarray(exp, dtype=np.uint8), coef=coef, xstar=None,
                  x0=np.stack([np.ones(n), np.zeros(n)], axis=-1), name=f"chandrasekhar{n}",
                  meta=dict(n=n, c=str(c)))


# -- batches of independent systems --------------------------------------------


@dataclass
class Batch:
    """Independent square systems stored back to back in sparse distributed form.

    System ``s`` owns polynomials ``[sys_poly[s], sys_poly[s+1])`` and
    variables ``[sys_var[s], sys_var[s+1])`` of the concatenated vectors;
    ``var`` holds variable indices local to each system.  The other arrays
    follow :class:`System`.
    """

    S: int
    sys_poly: np.ndarray  # int64 [S+1]
    sys_var: np.ndarray  # int64 [S+1]
    poly_ptr: np.ndarray  # int64 [P+1]
    mono_ptr: np.ndarray  # int64 [T+1]
    var: np.ndarray  # int32 [nnz], local
    exp: np.ndarray  # uint8 [nnz]
    coef: np.ndarray  # float64 [T, 2, 4]
    xstar: np.ndarray  # float64 [X, 2]
    x0: np.ndarray  # float64 [X, 2]
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> np.ndarray:
        return np.diff(self.sys_var)

    @property
    def T(self) -> int:
        return int(self.mono_ptr.shape[0] - 1)

    def point(self, which: str, L: int) -> np.ndarray:
        src = self.xstar if which == "xstar" else self.x0
        out = np.zeros((src.shape[0], 2, L), dtype=np.float64)
        out[:, :, 0] = src
        return out

    def system(self, s: int) -> System:
        """System ``s`` on its own (arrays rebased to start at 0)."""
        p0, p1 = int(self.sys_poly[s]), int(self.sys_poly[s + 1])
        t0, t1 = int(self.poly_ptr[p0]), int(self.poly_ptr[p1])
        o0, o1 = int(self.mono_ptr[t0]), int(self.mono_ptr[t1])
        v0, v1 = int(self.sys_var[s]), int(self.sys_var[s + 1])
        return System(N=p1 - p0, n=v1 - v0, poly_ptr=self.poly_ptr[p0:p1 + 1] - t0,
                      mono_ptr=self.mono_ptr[t0:t1 + 1] - o0, var=self.var[o0:o1].copy(),
                      exp=self.exp[o0:o1].copy(), coef=self.coef[t0:t1].copy(),
                      xstar=self.xstar[v0:v1].copy(), x0=self.x0[v0:v1].copy(),
                      name=f"batch[{s}]")


def _supports(rng, k, n):
    """Uniform k-subsets of range(n) (n <= 128) as 128-bit masks (lo, hi), one
    per entry of ``k``: Floyd's sampling, vectorised over the subsets."""
    T = k.shape[0]
    lo = np.zeros(T, dtype=np.uint64)
    hi = np.zeros(T, dtype=np.uint64)
    for i in range(int(k.max()) if T else 0):
        act = i < k
        j = n - k + i  # candidates [0, j]
        t = np.minimum((rng.random(T) * (j + 1)).astype(np.int64), j)
        sh = (t & 63).astype(np.uint64)
        up = t >= 64
        taken = np.where(up, hi >> sh, lo >> sh) & np.uint64(1)
        pick = np.where(taken.astype(bool), j, t)
        bit = np.left_shift(np.uint64(1), (pick & 63).astype(np.uint64)) * act.astype(np.uint64)
        up = pick >= 64
        hi |= np.where(up, bit, np.uint64(0))
        lo |= np.where(up, np.uint64(0), bit)
    return lo, hi


def _mask_bits(lo, hi, n):
    """(subset index, variable) pairs of the masks, variables ascending within a subset."""
    b = np.stack([lo, hi], axis=1).view(np.uint8).reshape(-1, 16)
    bits = np.unpackbits(b, axis=1, bitorder="little")[:, :n]
    t, v = np.nonzero(bits)
    return t, v.astype(np.int32)


def _mix(x):
    """64-bit mixing (splitmix64 finaliser) of uint64 arrays."""
    x = x.copy()
    x ^= x >> np.uint64(30)
    x *= np.uint64(0xBF58476D1CE4E5B9)
    x ^= x >> np.uint64(27)
    x *= np.uint64(0x94D049BB133111EB)
    x ^= x >> np.uint64(31)
    return x


def _exact_sums(values, starts):
    """Exact sums of the doubles ``values`` over the consecutive segments that
    begin at ``starts``, each rounded to a 4-limb nearest cascade.  Every
    double is split into four integer chunks on grids of 2^-40 .. 2^-160
    (exact for values of magnitude >= 2^-107, checked); chunk sums are exact
    in int64 (|chunk| < 2^41, fewer than 2^22 terms per segment) and are
    combined in Python integers."""
    rest = values.astype(np.float64)
    sums = []
    for c in range(4):
        q = np.trunc(np.ldexp(rest, 40 * (c + 1)))
        sums.append(np.add.reduceat(q.astype(np.int64), starts))
        rest = rest - np.ldexp(q, -40 * (c + 1))
    if np.any(rest != 0.0):
        raise ValueError("a term is not exact on the 2^-160 grid")
    out = np.zeros((starts.size, 4), dtype=np.float64)
    for i in range(starts.size):
        tot = (int(sums[0][i]) << 120) + (int(sums[1][i]) << 80) + (int(sums[2][i]) << 40) + int(sums[3][i])
        for l in range(4):  # nearest double of what is left (int -> float rounds to
            f = float(tot)  # nearest), then the exact remainder
            out[i, l] = math.ldexp(f, -160)
            tot -= int(f)
    return out


def _batch_system(n, seq, M_frac, k_max, dmax):
    """One system of a batch from its own seed sequence (see random_batch)."""
    r_sup, r_exp, r_coef, r_root, r_pert = [np.random.default_rng(q) for q in seq.spawn(5)]
    quarter = r_root.integers(0, 4, size=n)  # x*_j = i^quarter
    xstar = np.stack([np.array([1.0, 0.0, -1.0, 0.0])[quarter],
                      np.array([0.0, 1.0, 0.0, -1.0])[quarter]], axis=1)
    phi = 2.0 * math.pi * r_pert.random(n)
    x0 = xstar + 1e-6 * np.stack([np.cos(phi), np.sin(phi)], axis=-1)
    M = r_sup.integers(int(math.ceil(M_frac[0] * n)), int(math.floor(M_frac[1] * n)) + 1, size=n)
    Tm = int(M.sum())
    poly_of = np.repeat(np.arange(n), M)
    kk = r_sup.integers(2, min(k_max, n) + 1, size=Tm)
    lo, hi = _supports(r_sup, kk, n)
    emask = (np.left_shift(1, 2 * kk) - 1).astype(np.int64)
    ek = r_exp.integers(0, 1 << 32, size=Tm, dtype=np.int64) & emask
    for _ in range(100):  # distinct monomials within a polynomial: redraw duplicates
        h = _mix(_mix(_mix(lo ^ _mix(poly_of.astype(np.uint64))) ^ hi) ^ ek.astype(np.uint64))
        _, first = np.unique(h, return_index=True)
        dup = np.ones(Tm, dtype=bool)
        dup[first] = False
        if not dup.any():
            break
        idx = np.nonzero(dup)[0]
        lo[idx], hi[idx] = _supports(r_sup, kk[idx], n)
        ek[idx] = r_exp.integers(0, 1 << 32, size=idx.size, dtype=np.int64) & emask[idx]
    else:
        raise RuntimeError("could not draw distinct monomials")
    t_of, v = _mask_bits(lo, hi, n)
    slot = np.arange(t_of.size) - np.repeat(np.concatenate([[0], np.cumsum(kk)[:-1]]), kk)
    e = (((ek[t_of] >> (2 * slot)) & 3) % dmax + 1).astype(np.uint8)
    cth = 2.0 * math.pi * r_coef.random(Tm)
    c = np.stack([np.cos(cth), np.sin(cth)], axis=1)
    ph = np.zeros(Tm, dtype=np.int64)  # x*^a = i^ph
    np.add.at(ph, t_of, quarter[v] * e)
    ph %= 4
    re = np.choose(ph, [c[:, 0], -c[:, 1], -c[:, 0], c[:, 1]])
    im = np.choose(ph, [c[:, 1], c[:, 0], -c[:, 1], -c[:, 0]])
    starts = np.concatenate([[0], np.cumsum(M)[:-1]])
    const = np.stack([-_exact_sums(re, starts), -_exact_sums(im, starts)], axis=1)  # [n, 2, 4]
    return M, kk, v, e, c, const, xstar, x0


def _batch_chunk(args):
    ns, seqs, M_frac, k_max, dmax = args
    return [_batch_system(int(n), q, M_frac, k_max, dmax) for n, q in zip(ns, seqs)]


def random_batch(S: int, seed: int, n_range=(16, 128), M_frac=(0.5, 2.0), k_max: int = 16,
                 dmax: int = 4, workers: int = 0) -> Batch:
    """``S`` independent square systems (N = n).  n is uniform in ``n_range``;
    each polynomial has M uniform in [ceil(M_frac[0] n), floor(M_frac[1] n)]
    non-constant monomials plus a constant term; a monomial has k uniform in
    [2, min(k_max, n)] distinct variables (a uniform k-subset) with exponents
    uniform in 1..dmax (dmax <= 4); monomials within a polynomial are
    distinct; coefficients are unit-modulus.  The root x* has components in
    {1, i, -1, -i}, so each term c_t x*^a is the double c_t turned by a
    multiple of 90 degrees and the constant term -sum_t c_t x*^a is an exact
    sum of doubles, stored as a 4-limb cascade; x0 = x* + 1e-6 exp(i phi).
    System s draws from its own seed sequence (SeedSequence(seed).spawn(S)[s]),
    so it is the same whatever S' >= s+1 and however many worker processes
    (``workers``, spawned) build the batch."""
    if not 1 <= dmax <= 4:
        raise ValueError("dmax must be in 1..4")
    root = np.random.SeedSequence(seed)
    r_n = np.random.default_rng(root.spawn(1)[0])
    n_s = r_n.integers(n_range[0], n_range[1] + 1, size=S).astype(np.int64)
    seqs = np.random.SeedSequence(seed + (1 << 40)).spawn(S)
    if workers > 1 and S >= 64:
        import concurrent.futures as cf
        import multiprocessing as mp

        chunks = np.array_split(np.arange(S), workers * 4)
        jobs = [(n_s[c], [seqs[i] for i in c], M_frac, k_max, dmax) for c in chunks if c.size]
        with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            parts = [r for chunk in ex.map(_batch_chunk, jobs) for r in chunk]
    else:
        parts = _batch_chunk((n_s, seqs, M_frac, k_max, dmax))
    poly_ptr_l, mono_ptr_l, var_l, exp_l, coef_l = [np.zeros(1, np.int64)], [np.zeros(1, np.int64)], [], [], []
    xs_l, x0_l = [], []
    tcount = occ = 0
    for (M, kk, v, e, c, const, xstar, x0), n in zip(parts, n_s):
        n = int(n)
        Tm = int(M.sum())
        poly_of = np.repeat(np.arange(n), M)
        starts = np.concatenate([[0], np.cumsum(M)[:-1]])
        # per polynomial: its M monomials, then its constant term
        pos = np.arange(Tm) + poly_of
        cpos = starts + M + np.arange(n)
        klen = np.zeros(Tm + n, dtype=np.int64)
        klen[pos] = kk
        mono_ptr_l.append(occ + np.cumsum(klen))
        occ += int(kk.sum())
        poly_ptr_l.append(tcount + cpos + 1)
        cf_ = np.zeros((Tm + n, 2, 4), dtype=np.float64)
        cf_[pos, 0, 0] = c[:, 0]
        cf_[pos, 1, 0] = c[:, 1]
        cf_[cpos] = const
        coef_l.append(cf_)
        var_l.append(v)
        exp_l.append(e)
        xs_l.append(xstar)
        x0_l.append(x0)
        tcount += Tm + n
    sys_var = np.concatenate([[0], np.cumsum(n_s)]).astype(np.int64)
    return Batch(S=S, sys_poly=sys_var.copy(), sys_var=sys_var,
                 poly_ptr=np.concatenate(poly_ptr_l), mono_ptr=np.concatenate(mono_ptr_l),
                 var=np.concatenate(var_l).astype(np.int32), exp=np.concatenate(exp_l),
                 coef=np.concatenate(coef_l), xstar=np.concatenate(xs_l), x0=np.concatenate(x0_l),
                 meta=dict(S=S, seed=seed, n_range=n_range, M_frac=M_frac, k_max=k_max, dmax=dmax))


# -- named workloads ----------------------------------------------------------

WORKLOADS = {
    # plain Gauss-Newton, complex DD, 4 steps
    "gn32": dict(N=32, n=32, M=32, k=9, dmax=3, steps=4, config=1),
    # plain Gauss-Newton at scale (D, DD, QD)
    "gn256": dict(N=256, n=256, M=256, k=16, dmax=5, steps=4, config=2),
    # coefficient gradient at the converged root (complex DD)
    "adj128": dict(N=128, n=128, M=128, k=12, dmax=3, steps=4, config=4),
    # mixed precision: overdetermined and consistent, factorisation in double,
    # residuals in quad double (63 terms plus the constant per polynomial)
    "mix1536": dict(N=1536, n=1024, M=63, k=8, dmax=4, steps=4, config=5),
}

BATCH_WORKLOADS = {
    # batched Gauss-Newton, complex DD: 4096 systems, n in [16, 128]
    "batch4096": dict(S=4096, n_range=(16, 128), config=3),
}


@functools.lru_cache(maxsize=4)
def batch_workload(name: str, S: int | None = None, index: int = 0) -> Batch:
    """Named batch (cached); ``S`` overrides the number of systems (a prefix
    of the same stream of sizes is not kept: a different S draws afresh)."""
    import os

    w = BATCH_WORKLOADS[name]
    seed = BASE_SEED + 1000 * w["config"] + index
    S = w["S"] if S is None else S
    return random_batch(S, seed, n_range=w["n_range"], workers=min(16, os.cpu_count() or 1) if S >= 512 else 0)


@functools.lru_cache(maxsize=8)
def workload(name: str, system_index: int = 0) -> System:
    """Named workload (cached: callers must not modify the returned arrays)."""
    w = WORKLOADS[name]
    seed = BASE_SEED + 1000 * w["config"] + system_index
    return random_system(w["N"], w["n"], w["M"], w["k"], w["dmax"], seed, name=name)
