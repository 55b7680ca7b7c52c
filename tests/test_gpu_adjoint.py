"""GPU parity of the coefficient gradient (gn_adjoint) against the CPU oracle,
element by element, through the C ABI; the autograd wrapper and coefficient
updates on the device."""

import dataclasses

import numpy as np
import pytest

import oracle
from paper_1402_2626_gb300 import inputs
from tests._util import PARITY_TOL, limb_diff, term_scales

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = [("d", 1), ("dd", 2), ("qd", 4)]


def _gn():
    from paper_1402_2626_gb300 import build, gn

    build.build()
    return gn


def _root(s, L, steps=4):
    """The oracle's root of s from x0 at precision L."""
    x, _ = oracle.newton(s, s.point("x0", L), L, steps, nthreads=8)
    return x


def _gpu_adjoint(s, L, prec, x, arith="auto"):
    gn = _gn()
    sy = gn.System(s, arith=arith)
    xd = torch.tensor(x, device="cuda")
    gd = 2.0 * xd
    grad = torch.zeros((s.T, 2, L), dtype=torch.float64, device="cuda")
    lam = torch.zeros((s.N, 2, L), dtype=torch.float64, device="cuda")
    sy.adjoint(prec, xd, gd, grad, lam)
    out = grad.cpu().numpy(), lam.cpu().numpy()
    sy.close()
    return out


def _check(got, want, L, what):
    scale = float(np.abs(oracle.to_complex(want)).max())
    err = limb_diff(got, want)
    assert err.max() <= PARITY_TOL[L] * scale, (what, float(err.max()), scale)


SMALL = [
    ("square", dict(N=24, n=24, M=(12, 30), k=(1, 6), dmax=3, seed=501)),
    ("overdetermined ragged", dict(N=45, n=30, M=(10, 20), k=(1, 5), dmax=3, seed=502)),
    # three 16-column blocks, the last partial: the blocked forward substitution
    ("blocked ragged", dict(N=50, n=40, M=(10, 20), k=(1, 5), dmax=3, seed=507)),
]


@pytest.mark.parametrize("arith", ["auto", "int", "fp64"])
@pytest.mark.parametrize("prec,L", PRECS)
@pytest.mark.parametrize("name,kw", SMALL, ids=[c[0] for c in SMALL])
def test_adjoint_parity_small(name, kw, prec, L, arith):
    s = inputs.random_system(kw["N"], kw["n"], kw["M"], kw["k"], kw["dmax"], seed=kw["seed"])
    x = _root(s, L)
    grad_o, lam_o = oracle.adjoint(s, x, 2.0 * x, L, nthreads=8)
    grad, lam = _gpu_adjoint(s, L, prec, x, arith)
    _check(grad, grad_o, L, "grad")
    _check(lam, lam_o, L, "lambda")


@pytest.mark.parametrize("arith", ["auto", "fp64"])
@pytest.mark.parametrize("prec,L", PRECS)
def test_adjoint_reuse_last_step(prec, L, arith):
    """GN_ADJ_REUSE after a Newton step from a converged point: the gradient
    at the new iterate from the step's own factorisation matches the oracle
    (which factors J at that iterate); a second reuse gives the same; after
    gn_system_set_coef there is nothing to reuse."""
    gn = _gn()
    name, kw = SMALL[1]
    s = inputs.random_system(kw["N"], kw["n"], kw["M"], kw["k"], kw["dmax"], seed=kw["seed"])
    x = _root(s, L)
    sy = gn.System(s, arith=arith)
    xd = torch.tensor(x, device="cuda")
    sy.newton(prec, xd, 1)
    gd = 2.0 * xd
    grad = torch.zeros((s.T, 2, L), dtype=torch.float64, device="cuda")
    lam = torch.zeros((s.N, 2, L), dtype=torch.float64, device="cuda")
    sy.adjoint(prec, xd, gd, grad, lam, reuse=True)
    g1 = grad.cpu().numpy()
    xh = xd.cpu().numpy()
    grad_o, lam_o = oracle.adjoint(s, xh, 2.0 * xh, L, nthreads=8)
    _check(g1, grad_o, L, "grad")
    _check(lam.cpu().numpy(), lam_o, L, "lambda")
    grad.zero_()
    sy.adjoint(prec, xd, gd, grad, reuse=True)
    assert np.array_equal(grad.cpu().numpy(), g1)
    sy.set_coef(torch.tensor(s.coef[:, :, :L], device="cuda"))
    with pytest.raises(gn.GnError) as ei:
        sy.adjoint(prec, xd, gd, grad, reuse=True)
    assert ei.value.status == 1
    sy.close()


def test_adjoint_empty_polynomial():
    """A polynomial without terms (a zero row of J, lambda_i = 0) between
    others: the term-to-polynomial search must skip it."""
    s = inputs.random_system(8, 5, (3, 6), (1, 3), 3, seed=503)
    pp = np.insert(s.poly_ptr, 3, s.poly_ptr[3])  # polynomial 3 becomes empty
    s = dataclasses.replace(s, N=s.N + 1, poly_ptr=pp)
    L = 2
    x = _root(s, L)
    grad_o, lam_o = oracle.adjoint(s, x, 2.0 * x, L)
    grad, lam = _gpu_adjoint(s, L, "dd", x)
    assert not np.any(lam[3])
    _check(grad, grad_o, L, "grad")
    _check(lam, lam_o, L, "lambda")


def test_adjoint_singular_reports():
    """A Jacobian column that vanishes at x: GN_ESINGULAR, not a gradient."""
    gn = _gn()
    s = inputs.random_system(6, 4, (3, 5), (1, 3), 3, seed=504)
    coef = s.coef.copy()
    for t in range(s.T):
        a, b = int(s.mono_ptr[t]), int(s.mono_ptr[t + 1])
        if np.any(s.var[a:b] == 2):
            coef[t] = 0.0
    s = dataclasses.replace(s, coef=coef)
    sy = gn.System(s)
    x = torch.tensor(s.point("xstar", 2), device="cuda")
    grad = torch.zeros((s.T, 2, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(gn.GnError) as ei:
        sy.adjoint("dd", x, 2.0 * x, grad)
    assert ei.value.status == 4
    sy.close()


def test_adjoint_full_size_dd():
    """The 128-variable workload (N = n = 128, 128 terms of 12 variables per
    polynomial, exponents 1..3, complex DD): Newton on the GPU from x0, then
    every one of the 16,512 gradients against the oracle at the same root."""
    gn = _gn()
    s = inputs.workload("adj128")
    L = 2
    sy = gn.System(s)
    x = torch.tensor(s.point("x0", L), device="cuda")
    rep = sy.newton("dd", x, 4)
    assert rep["dx_norm"][-1] < 1e-28
    grad = torch.zeros((s.T, 2, L), dtype=torch.float64, device="cuda")
    lam = torch.zeros((s.N, 2, L), dtype=torch.float64, device="cuda")
    sy.adjoint("dd", x, 2.0 * x, grad, lam)
    xh = x.cpu().numpy()
    grad_o, lam_o = oracle.adjoint(s, xh, 2.0 * xh, L, nthreads=16)
    _check(grad.cpu().numpy(), grad_o, L, "grad")
    _check(lam.cpu().numpy(), lam_o, L, "lambda")
    # the factorisation of the last Newton step gives the same at DD accuracy
    x.copy_(torch.tensor(s.point("x0", L), device="cuda"))
    sy.newton("dd", x, 4)
    assert np.array_equal(x.cpu().numpy(), xh)
    sy.adjoint("dd", x, 2.0 * x, grad, lam, reuse=True)
    _check(grad.cpu().numpy(), grad_o, L, "grad (reuse)")
    sy.close()


def test_set_coef_then_eval():
    """Coefficients replaced on the device are the ones the next evaluation uses."""
    gn = _gn()
    s = inputs.random_system(10, 8, (4, 8), (1, 4), 3, seed=505)
    L = 2
    sy = gn.System(s)
    rng = np.random.default_rng(7)
    coef2 = s.coef.copy()
    coef2[:, :, 0] += rng.normal(size=(s.T, 2)) * 0.25
    coef2[:, :, 1] = 0.0
    coef2[:, :, 1] = rng.normal(size=(s.T, 2)) * 1e-18 * np.abs(coef2[:, :, 0])
    coef2[:, :, L:] = 0.0  # the device holds L limbs: the oracle evaluates the same values
    s2 = dataclasses.replace(s, coef=coef2)
    sy.set_coef(torch.tensor(coef2[:, :, :L], device="cuda"))
    x = torch.tensor(s.point("x0", L), device="cuda")
    f = torch.zeros((s.N, 2, L), dtype=torch.float64, device="cuda")
    J = torch.zeros((s.n, s.N, 2, L), dtype=torch.float64, device="cuda")
    sy.eval("dd", x, f, J)
    fo, Jo, _ = oracle.evaluate(s2, s.point("x0", L), L)
    # the stated tolerance per entry, scaled by the entry's term magnitudes
    Sf, SJ = term_scales(s2, s.point("x0", L))
    assert np.all(limb_diff(f.cpu().numpy(), fo) <= PARITY_TOL[L] * Sf)
    assert np.all(limb_diff(J.cpu().numpy().transpose(1, 0, 2, 3), Jo) <= PARITY_TOL[L] * SJ)
    sy.close()


def test_autograd_newton_root():
    """torch.autograd through newton_root: loss = sum |x|^2 on the leading
    limbs; dL/dcoef equals the oracle's gradient for g = 2 x_0 in every limb."""
    gn = _gn()
    s = inputs.random_system(16, 16, (8, 16), (1, 4), 3, seed=506)
    L = 2
    sy = gn.System(s)
    coef = torch.tensor(s.coef[:, :, :L], device="cuda", requires_grad=True)
    x0 = torch.tensor(s.point("x0", L), device="cuda")
    x = gn.newton_root(sy, "dd", coef, x0, 4)
    loss = (x[..., 0] ** 2).sum()
    loss.backward()
    xh = x.detach().cpu().numpy()
    g = np.zeros_like(xh)
    g[..., 0] = 2.0 * xh[..., 0]
    grad_o, _ = oracle.adjoint(s, xh, g, L)
    gc = coef.grad.cpu().numpy()
    assert np.array_equal(gc[..., 0], gc[..., 1])
    want = oracle.to_complex(grad_o)
    got = gc[..., 0, 0] + 1j * gc[..., 1, 0]
    assert np.abs(got - want).max() <= 1e-15 * np.abs(want).max()
    # the root itself is the oracle's Newton result
    xo, _ = oracle.newton(s, s.point("x0", L), L, 4)
    assert limb_diff(xh, xo).max() <= PARITY_TOL[L]
    sy.close()
