"""GPU parity of gn_eval (Section 2) against the CPU oracle.

Every case calls the CUDA library through the C ABI and compares f and J
entry by entry with the oracle on the same seeded inputs, at
|gpu - oracle| <= tol_L * S where S is the sum of the magnitudes of the terms
that make up the entry (tol = 1e-13, 1e-26, 1e-58 for D, DD, QD).
"""

import numpy as np
import pytest

import oracle
from paper_1402_2626_gb300 import inputs
from tests._util import PARITY_TOL, limb_diff, term_scales

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = [("d", 1), ("dd", 2), ("qd", 4)]
# integer-mantissa evaluation (default) and FP64 error-free transformations
ARITHS = ["int", "fp64"]


def _gn():
    from paper_1402_2626_gb300 import build, gn

    build.build()
    return gn


def gpu_eval(system, x, L, prec, arith="int"):
    gn = _gn()
    s = gn.System(system, arith=arith)
    xd = torch.tensor(np.ascontiguousarray(x[..., :L]), device="cuda")
    f = torch.full((system.N, 2, L), np.nan, dtype=torch.float64, device="cuda")
    J = torch.full((system.n, system.N, 2, L), np.nan, dtype=torch.float64, device="cuda")
    s.eval(prec, xd, f, J)
    torch.cuda.synchronize()
    out = f.cpu().numpy(), J.cpu().numpy().transpose(1, 0, 2, 3)
    s.close()
    return out


def check(system, x, L, prec, rows=None, arith="int"):
    f, J = gpu_eval(system, x, L, prec, arith)
    r0, r1 = (0, system.N) if rows is None else rows
    fo, Jo, _ = oracle.evaluate(system, x, L, "reverse", rows=(r0, r1), nthreads=8)
    Sf, SJ = term_scales(system, x, rows=(r0, r1))
    tol = PARITY_TOL[L]
    ef = limb_diff(f[r0:r1], fo)
    eJ = limb_diff(J[r0:r1], Jo)
    assert np.all(ef <= tol * Sf), (prec, float((ef / np.maximum(Sf, 1e-300)).max()))
    # entries no term touches must be exactly zero
    zero = SJ == 0
    assert not np.any(J[r0:r1][zero]), "structural zeros must be 0"
    assert np.all(eJ[~zero] <= tol * SJ[~zero]), (prec, float((eJ[~zero] / SJ[~zero]).max()))
    return float((ef / np.maximum(Sf, 1e-300)).max()), float((eJ[~zero] / SJ[~zero]).max())


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("prec,L", PRECS)
def test_edge_cases(prec, L, arith):
    # one variable; constant-only polynomial; k = 1; a variable in no term
    # (zero column); long supports (k up to 40) and high exponents (7)
    cases = [
        inputs.random_system(1, 1, 3, 1, 7, seed=1),
        inputs.random_system(3, 3, (1, 4), (1, 3), 4, seed=2, constant=False),
        inputs.random_system(6, 5, (0, 3), (1, 5), 3, seed=3),
        inputs.random_system(48, 48, 2, (30, 40), 3, seed=4),
        inputs.random_system(5, 4, 6, 1, 5, seed=5),
    ]
    # a variable that appears in no term: a zero Jacobian column
    s = inputs.random_system(5, 4, 4, (1, 3), 3, seed=6)
    x5 = np.vstack([s.x0, [[0.6, 0.8]]])
    cases.append(inputs.System(N=5, n=5, poly_ptr=s.poly_ptr, mono_ptr=s.mono_ptr, var=s.var,
                               exp=s.exp, coef=s.coef, xstar=x5, x0=x5))
    for sys_ in cases:
        x = sys_.point("x0", L)
        check(sys_, x, L, prec, arith=arith)


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("prec,L", PRECS)
def test_support_length_boundaries(prec, L, arith):
    """Supports of exactly k variables around the per-thread limit (64, above
    which a warp takes a term) and around multiples of the warp's 32 lanes,
    with exponents up to 3 (common factors inside long supports)."""
    for k in (31, 32, 33, 63, 64, 65, 66, 95, 96, 97, 127, 128, 129, 200):
        n = k + 8
        sys_ = inputs.random_system(n, n, 2, k, 3, seed=1000 + k)
        check(sys_, sys_.point("x0", L), L, prec, arith=arith)


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("prec,L", PRECS)
def test_gn32_full(prec, L, arith):
    s = inputs.workload("gn32")
    check(s, s.point("x0", L), L, prec, arith=arith)


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("prec,L", PRECS)
def test_ragged_many_tiles(prec, L, arith):
    # T not a multiple of the 128-thread CTA, N not a multiple of 4 warps
    s = inputs.random_system(37, 29, (20, 45), (1, 14), 5, seed=77)
    check(s, s.point("x0", L), L, prec, arith=arith)


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("prec,L", PRECS)
def test_gn256_sampled_rows(prec, L, arith):
    """Full-size workload (n = N = 256, 256 terms of 16 variables per
    polynomial, exponents 1..5), sampled rows checked one by one."""
    s = inputs.workload("gn256")
    x = s.point("x0", L)
    f, J = gpu_eval(s, x, L, prec, arith)
    tol = PARITY_TOL[L]
    for i in (0, 1, 127, 200, 255):
        fo, Jo, _ = oracle.evaluate(s, x, L, "reverse", rows=(i, i + 1), nthreads=8)
        Sf, SJ = term_scales(s, x, rows=(i, i + 1))
        assert np.all(limb_diff(f[i:i + 1], fo) <= tol * Sf)
        nz = SJ > 0
        assert np.all(limb_diff(J[i:i + 1], Jo)[nz] <= tol * SJ[nz])
        assert not np.any(J[i:i + 1][~nz])


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("prec,L", PRECS)
def test_deterministic(prec, L, arith):
    s = inputs.random_system(16, 16, 20, (2, 9), 4, seed=9)
    a = gpu_eval(s, s.point("x0", L), L, prec, arith)
    b = gpu_eval(s, s.point("x0", L), L, prec, arith)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("arith", ARITHS)
def test_root_residual_dd(arith):
    """At the built-in root f vanishes to DD level (Section 5 setting)."""
    s = inputs.workload("gn32")
    f, _ = gpu_eval(s, s.point("xstar", 2), 2, "dd", arith)
    Sf, _ = term_scales(s, s.point("xstar", 2))
    assert np.all(limb_diff(f, np.zeros_like(f)) <= 1e-28 * Sf)


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("prec,L", PRECS)
def test_f_alone_equals_f_with_j(prec, L, arith):
    """An evaluation of f without J (the mixed solver's refinement steps)
    forms each term's value alone; it must give the same f, bit for bit, as
    the evaluation that also forms J, with supports short (one lane per
    term), longer than 16 and longer than 64 (a warp per term), and match
    the oracle."""
    gn = _gn()
    for seed, (N, n, M, k, dmax) in enumerate([(37, 29, (20, 45), (1, 14), 5), (48, 40, (3, 8), (17, 40), 4),
                                               (72, 72, 2, (60, 70), 3)]):
        system = inputs.random_system(N, n, M, k, dmax, seed=300 + seed)
        x = system.point("x0", L)
        s = gn.System(system, arith=arith)
        xd = torch.tensor(np.ascontiguousarray(x[..., :L]), device="cuda")
        f0 = torch.full((N, 2, L), np.nan, dtype=torch.float64, device="cuda")
        f1 = torch.full((N, 2, L), np.nan, dtype=torch.float64, device="cuda")
        J = torch.full((n, N, 2, L), np.nan, dtype=torch.float64, device="cuda")
        s.eval(prec, xd, f0, J)
        s.eval(prec, xd, f1, None)
        torch.cuda.synchronize()
        a, b = f0.cpu().numpy(), f1.cpu().numpy()
        assert np.array_equal(a, b), (seed, float(np.nanmax(np.abs(a - b))))
        fo, _, _ = oracle.evaluate(system, x, L, "reverse", jacobian=False, nthreads=8)
        Sf, _ = term_scales(system, x)
        assert np.all(limb_diff(b, fo) <= PARITY_TOL[L] * Sf)
        s.close()
