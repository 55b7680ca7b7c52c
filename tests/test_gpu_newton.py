"""GPU parity of the least-squares solver (Section 3) and of Gauss-Newton
(Section 4) against the CPU oracle, through the C ABI."""

import numpy as np
import pytest

import oracle
from paper_1402_2626_gb300 import inputs
from tests._util import PARITY_TOL, limb_diff, lstsq_sensitivity, term_scales

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = [("d", 1), ("dd", 2), ("qd", 4)]
# integer mantissas (default) and FP64 error-free transformations
ARITHS = ["int", "fp64"]


def _gn():
    from paper_1402_2626_gb300 import build, gn

    build.build()
    return gn


def _rand_matrix(rng, m, ncols, L):
    A = np.zeros((m, ncols, 2, L))
    A[..., 0, 0] = rng.standard_normal((m, ncols))
    A[..., 1, 0] = rng.standard_normal((m, ncols))
    if L > 1:
        A[..., :, 1] = A[..., :, 0] * 2.0 ** -55 * rng.standard_normal((m, ncols, 2))
    return A


def gpu_lstsq(A, L, prec, arith="int"):
    gn = _gn()
    m, ncols = A.shape[0], A.shape[1]
    # any system provides the workspace handle
    s = gn.System(inputs.random_system(2, 2, 2, 1, 1, seed=0), arith=arith)
    Ab = torch.tensor(np.ascontiguousarray(A.transpose(1, 0, 2, 3)), device="cuda")
    R = torch.zeros((ncols, ncols, 2, L), dtype=torch.float64, device="cuda")
    dx = torch.zeros((ncols - 1, 2, L), dtype=torch.float64, device="cuda")
    try:
        s.lstsq(prec, Ab, R, dx)
    finally:
        torch.cuda.synchronize()
        s.close()
    return (Ab.cpu().numpy().transpose(1, 0, 2, 3), R.cpu().numpy().transpose(1, 0, 2, 3),
            dx.cpu().numpy())


def _check_lstsq(R, Q, dx, Ro, Qo, dxo, tol, kappa, cn, fx, n):
    """GPU against oracle within the first-order perturbation bounds of the
    case (tests._util.lstsq_sensitivity) with eps = the stated tolerance."""
    eR = limb_diff(R, Ro) / (tol * kappa * cn[None, :])
    assert eR.max() <= 1.0, ("R", float(eR.max()), kappa)
    assert not np.any(np.tril(np.ones((n + 1, n + 1)), -1)[..., None, None] * R)
    eQ = limb_diff(Q[:, :n], Qo[:, :n]) / (tol * kappa)
    assert eQ.max() <= 1.0, ("Q", float(eQ.max()), kappa)
    if dx is not None:
        ex = limb_diff(dx, dxo) / (tol * fx)
        assert ex.max() <= 1.0, ("dx", float(ex.max()), kappa, fx)


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("prec,L", PRECS)
@pytest.mark.parametrize("m,n", [(1, 1), (7, 4), (40, 33), (130, 127), (300, 257), (513, 60)])
def test_lstsq_parity(prec, L, m, n, arith):
    rng = np.random.default_rng(m * 1000 + n)
    A = _rand_matrix(rng, m, n + 1, L)
    Q, R, dx = gpu_lstsq(A, L, prec, arith)
    Qo, Ro = oracle.mgs(A, L, nthreads=8)
    dxo = oracle.backsub(Ro, L)
    tol = PARITY_TOL[L]
    kappa, cn, fx = lstsq_sensitivity(A, Ro)
    _check_lstsq(R, Q, dx, Ro, Qo, dxo, tol, kappa, cn, fx, n)


@pytest.mark.parametrize("prec,L", PRECS)
def test_lstsq_parity_two_rows_per_thread(prec, L):
    """n = 600 > 512: back substitution with two rows per thread."""
    rng = np.random.default_rng(600)
    m, n = 620, 600
    A = _rand_matrix(rng, m, n + 1, L)
    Q, R, dx = gpu_lstsq(A, L, prec)
    Qo, Ro = oracle.mgs(A, L, nthreads=16)
    dxo = oracle.backsub(Ro, L)
    tol = PARITY_TOL[L]
    kappa, cn, fx = lstsq_sensitivity(A, Ro)
    _check_lstsq(R, Q, dx, Ro, Qo, dxo, tol, kappa, cn, fx, n)


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("prec,L", PRECS)
@pytest.mark.parametrize("m,n", [(40, 33), (256, 256)])
def test_mgs_factorisation_only(prec, L, m, n, arith):
    """gn_mgs: the factorisation of gn_lstsq, asynchronous, status on the device."""
    gn = _gn()
    rng = np.random.default_rng(m * 7 + n)
    A = _rand_matrix(rng, m, n + 1, L)
    s = gn.System(inputs.random_system(n, n, 2, 1, 1, seed=0), arith=arith)
    Ab = torch.tensor(np.ascontiguousarray(A.transpose(1, 0, 2, 3)), device="cuda")
    R = torch.zeros((n + 1, n + 1, 2, L), dtype=torch.float64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    s.mgs(prec, Ab, R, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Q, Rg = Ab.cpu().numpy().transpose(1, 0, 2, 3), R.cpu().numpy().transpose(1, 0, 2, 3)
    Qo, Ro = oracle.mgs(A, L, nthreads=8)
    tol = PARITY_TOL[L]
    kappa, cn, _ = lstsq_sensitivity(A, Ro)
    _check_lstsq(Rg, Q, None, Ro, Qo, None, tol, kappa, cn, 0.0, n)
    # a repeated column: the status word reports the rank deficiency
    A[:, 2] = A[:, 0]
    Ab.copy_(torch.tensor(np.ascontiguousarray(A.transpose(1, 0, 2, 3))))
    s.mgs(prec, Ab, R, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 4
    s.close()


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("prec,L", PRECS)
def test_lstsq_singular(prec, L, arith):
    gn = _gn()
    rng = np.random.default_rng(5)
    A = _rand_matrix(rng, 9, 5, L)
    A[:, 2] = A[:, 0]
    with pytest.raises(gn.GnError) as e:
        gpu_lstsq(A, L, prec, arith)
    assert e.value.status == 4


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("prec,L", PRECS)
def test_newton_gn32_parity(prec, L, arith):
    """Four steps from x* + 1e-6 (the plain Gauss-Newton workload): the GPU
    iterates match the oracle's and converge quadratically to x*."""
    gn = _gn()
    s = inputs.workload("gn32")
    sysg = gn.System(s, arith=arith)
    x = torch.tensor(s.point("x0", L), device="cuda")
    xo = s.point("x0", L)
    tol = PARITY_TOL[L]
    errs = []
    for step in range(4):
        rep = sysg.newton(prec, x, 1)
        assert rep["steps_done"] == 1
        xo_prev = xo
        xo, dxo, fo, _ = oracle.newton_step(s, xo, L, nthreads=8)
        xg = x.cpu().numpy()
        assert np.all(limb_diff(xg, xo) <= tol), (step, float(limb_diff(xg, xo).max()))
        d = xg.copy()
        d[:, :, 0] -= s.xstar
        errs.append(float(limb_diff(d, np.zeros_like(d)).max()))
        fo_norm = float(np.sqrt((fo[:, :, 0] ** 2).sum()))
        # | ||f_gpu|| - ||f_o|| | <= ||f_gpu - f_o|| <= tol ||S_f|| (per-entry
        # parity), plus the rounding of a double norm over N entries
        Sf, _ = term_scales(s, xo_prev)
        bound = (s.N + 2) * 2.0 ** -52 * fo_norm + tol * float(np.linalg.norm(Sf))
        assert abs(rep["res_norm"][0] - fo_norm) <= bound
    assert errs[-1] <= tol
    assert errs[1] <= max(1e4 * errs[0] ** 2, tol)
    sysg.close()


@pytest.mark.parametrize("prec,L", PRECS)
def test_newton_multi_step_report(prec, L):
    gn = _gn()
    s = inputs.workload("gn32")
    sysg = gn.System(s)
    x = torch.tensor(s.point("x0", L), device="cuda")
    rep = sysg.newton(prec, x, 4)
    assert rep["steps_done"] == 4
    # quadratic contraction of the residual until the precision floor
    r = rep["res_norm"]
    assert r[1] <= 100 * r[0] ** 2 + 1e-12
    xo, _ = oracle.newton(s, s.point("x0", L), L, 4, nthreads=8)
    assert np.all(limb_diff(x.cpu().numpy(), xo) <= PARITY_TOL[L])
    # tolerance-driven stop
    x2 = torch.tensor(s.point("x0", L), device="cuda")
    rep2 = sysg.newton(prec, x2, 10, tol=1e-8)
    assert rep2["status"] == 0 and rep2["steps_done"] <= 4
    sysg.close()


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("prec,L", PRECS)
def test_newton_gn256_step_parity(prec, L, arith):
    """One full-size step (n = N = 256, 65,792 terms) in D, DD and QD: every
    component of the new iterate against the oracle's step."""
    gn = _gn()
    s = inputs.workload("gn256")
    sysg = gn.System(s, arith=arith)
    x = torch.tensor(s.point("x0", L), device="cuda")
    sysg.newton(prec, x, 1)
    xo, _, _, _ = oracle.newton_step(s, s.point("x0", L), L, nthreads=16)
    err = limb_diff(x.cpu().numpy(), xo)
    assert np.all(err <= PARITY_TOL[L]), float(err.max())
    sysg.close()


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("prec,L", PRECS)
def test_newton_gn256_converges(prec, L, arith):
    """Property at full size: quadratic convergence to the built-in root."""
    gn = _gn()
    s = inputs.workload("gn256")
    sysg = gn.System(s, arith=arith)
    x = torch.tensor(s.point("x0", L), device="cuda")
    rep = sysg.newton(prec, x, 4)
    d = x.cpu().numpy()
    d[:, :, 0] -= s.xstar
    err = float(limb_diff(d, np.zeros_like(d)).max())
    assert err <= PARITY_TOL[L], (prec, err, rep)
    sysg.close()


def test_newton_singular_reports():
    """A variable that appears in no term gives a zero Jacobian column, which
    the rank test of the first pivot beyond it reports as GN_ESINGULAR."""
    gn = _gn()
    base = inputs.random_system(6, 4, 6, (1, 3), 3, seed=8)
    x5 = np.vstack([base.x0, [[0.6, 0.8]]])
    bad = inputs.System(N=6, n=5, poly_ptr=base.poly_ptr, mono_ptr=base.mono_ptr, var=base.var,
                        exp=base.exp, coef=base.coef, xstar=x5, x0=x5)
    sysg = gn.System(bad)
    x = torch.tensor(bad.point("x0", 2), device="cuda")
    x_before = x.clone()
    rep = sysg.newton("dd", x, 3, raise_on_error=False)
    assert rep["status"] == 4 and rep["steps_done"] == 0
    assert torch.equal(x, x_before)  # no update was applied
    sysg.close()


def test_arith_switch_rebuilds_step():
    """Switching the arithmetic between runs on the same x pointer discards
    the captured step: each run matches the oracle's iterates."""
    gn = _gn()
    L = 2
    s = inputs.workload("gn32")
    sysg = gn.System(s)
    x = torch.tensor(s.point("x0", L), device="cuda")
    xo = s.point("x0", L)
    for arith in ("auto", "int", "fp64", "auto"):
        sysg.set_arith(arith)
        sysg.newton("dd", x, 1)
        xo, _, _, _ = oracle.newton_step(s, xo, L, nthreads=8)
        assert np.all(limb_diff(x.cpu().numpy(), xo) <= PARITY_TOL[L]), arith
    assert sysg._lib.gn_system_set_arith(sysg._h, 7) == 1  # unknown value: GN_EINVAL
    assert sysg._lib.gn_system_set_arith(sysg._h, -1) == 1
    sysg.close()
