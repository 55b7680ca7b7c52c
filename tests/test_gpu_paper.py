"""GPU parity on the paper's benchmark systems (Section 5) against the CPU
oracle: evaluation and differentiation of cyclic n-roots (supports up to n
variables, the warp-per-term kernel beyond 64), Newton's method on its
homotopy f(x) - t f(z), and Newton's method on the Chandrasekhar H-equation."""

import numpy as np
import pytest

import oracle
from paper_1402_2626_gb300 import inputs
from tests._util import PARITY_TOL, limb_diff, rounding_residual_scale, term_scales

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = [("d", 1), ("dd", 2), ("qd", 4)]


def _gn():
    from paper_1402_2626_gb300 import build, gn

    build.build()
    return gn


def _eval_gpu(sy, s, prec, L, x):
    xd = torch.tensor(x, device="cuda")
    f = torch.zeros((s.N, 2, L), dtype=torch.float64, device="cuda")
    J = torch.zeros((s.n, s.N, 2, L), dtype=torch.float64, device="cuda")
    sy.eval(prec, xd, f, J)
    return f.cpu().numpy(), J.cpu().numpy().transpose(1, 0, 2, 3)


@pytest.mark.parametrize("prec,L", PRECS)
@pytest.mark.parametrize("n", [70, 130])
def test_cyclic_eval_parity(n, prec, L):
    gn = _gn()
    s = inputs.cyclic(n, seed=1)
    x = s.point("x0", L)
    sy = gn.System(s)
    f, J = _eval_gpu(sy, s, prec, L, x)
    fo, Jo, _ = oracle.evaluate(s, x, L, nthreads=16)
    Sf, SJ = term_scales(s, x)
    assert np.all(limb_diff(f, fo) <= PARITY_TOL[L] * Sf)
    assert np.all(limb_diff(J, Jo) <= PARITY_TOL[L] * np.maximum(SJ, 1e-300))
    sy.close()


def test_cyclic512_eval_sampled_rows():
    """Cyclic 512-roots in DD (supports up to 512): sampled rows of f and J
    against the oracle's evaluation of those rows."""
    gn = _gn()
    n, L = 512, 2
    s = inputs.cyclic(n, seed=2)
    x = s.point("x0", L)
    sy = gn.System(s)
    f, J = _eval_gpu(sy, s, "dd", L, x)
    for rows in ((0, 2), (63, 66), (300, 301), (509, 512)):
        fo, Jo, _ = oracle.evaluate(s, x, L, rows=rows, nthreads=16)
        Sf, SJ = term_scales(s, x, rows=rows)
        assert np.all(limb_diff(f[rows[0]:rows[1]], fo) <= PARITY_TOL[L] * Sf), rows
        assert np.all(limb_diff(J[rows[0]:rows[1]], Jo) <= PARITY_TOL[L] * np.maximum(SJ, 1e-300)), rows
    sy.close()


@pytest.mark.parametrize("prec,L", [("dd", 2), ("qd", 4)])
def test_cyclic_homotopy_newton_parity(prec, L):
    """Newton's method on f(x) - t f(z) from z (Section 5.3) at n = 80:
    every iterate equals the oracle's."""
    gn = _gn()
    s = inputs.cyclic_homotopy(80, seed=4)
    sy = gn.System(s)
    x = torch.tensor(s.point("x0", L), device="cuda")
    xo = s.point("x0", L)
    for step in range(4):
        sy.newton(prec, x, 1)
        xo, _, _, _ = oracle.newton_step(s, xo, L, nthreads=16)
        assert limb_diff(x.cpu().numpy(), xo).max() <= PARITY_TOL[L], step
    sy.close()


def test_cyclic512_homotopy_newton_dd():
    """The paper's closing experiment (Section 5.3): Newton's method on the
    homotopy of cyclic 512-roots in complex DD from z; seven iterations reach
    the full precision (||dx|| at the DD floor); residuals of sampled rows,
    evaluated by the oracle at the GPU's x, are within the residual that a
    root accurate to the stated DD tolerance in every component leaves."""
    gn = _gn()
    s = inputs.cyclic_homotopy(512, seed=0)
    sy = gn.System(s)
    x = torch.tensor(s.point("x0", 2), device="cuda")
    rep = sy.newton("dd", x, 7)
    assert rep["dx_norm"][-1] < 1e-25 * rep["dx_norm"][0]
    xh = x.cpu().numpy()
    for rows in ((0, 1), (255, 256), (510, 512)):
        f, _, _ = oracle.evaluate(s, xh, 2, rows=rows, jacobian=False, nthreads=16)
        scale = rounding_residual_scale(s, xh, rows=rows)
        assert np.all(limb_diff(f, np.zeros_like(f)) <= PARITY_TOL[2] * scale), rows
    sy.close()


@pytest.mark.parametrize("prec,L", PRECS)
def test_chandrasekhar_newton_parity(prec, L):
    gn = _gn()
    s = inputs.chandrasekhar(64)
    sy = gn.System(s)
    x = torch.tensor(s.point("x0", L), device="cuda")
    sy.newton(prec, x, 6)
    xo, _ = oracle.newton(s, s.point("x0", L), L, 6, nthreads=16)
    assert limb_diff(x.cpu().numpy(), xo).max() <= PARITY_TOL[L]
    sy.close()


def test_chandrasekhar1024_dd():
    """Six Newton iterations in complex DD at n = 1024 from H = 1 (Table 3's
    setting): quadratic convergence and residuals of sampled rows at the DD
    rounding level of their terms."""
    gn = _gn()
    s = inputs.chandrasekhar(1024)
    sy = gn.System(s)
    x = torch.tensor(s.point("x0", 2), device="cuda")
    rep = sy.newton("dd", x, 6)
    dx = rep["dx_norm"]
    assert dx[-1] < 1e-28
    xh = x.cpu().numpy()
    assert np.all(xh[:, 0, 0] > 1.0) and np.all(xh[:, 0, 0] < 2.0)  # the positive solution near 1
    for rows in ((0, 4), (1020, 1024)):
        f, _, _ = oracle.evaluate(s, xh, 2, rows=rows, jacobian=False, nthreads=16)
        Sf, _ = term_scales(s, xh, rows=rows)
        assert np.all(limb_diff(f, np.zeros_like(f)) <= PARITY_TOL[2] * Sf), rows
    sy.close()
