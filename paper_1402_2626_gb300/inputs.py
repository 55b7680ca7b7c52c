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


# -- named workloads ----------------------------------------------------------

WORKLOADS = {
    # plain Gauss-Newton, complex DD, 4 steps
    "gn32": dict(N=32, n=32, M=32, k=9, dmax=3, steps=4, config=1),
    # plain Gauss-Newton at scale (D, DD, QD)
    "gn256": dict(N=256, n=256, M=256, k=16, dmax=5, steps=4, config=2),
}


@functools.lru_cache(maxsize=8)
def workload(name: str, system_index: int = 0) -> System:
    """Named workload (cached: callers must not modify the returned arrays)."""
    w = WORKLOADS[name]
    seed = BASE_SEED + 1000 * w["config"] + system_index
    return random_system(w["N"], w["n"], w["M"], w["k"], w["dmax"], seed, name=name)
