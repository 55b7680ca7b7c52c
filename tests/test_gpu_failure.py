"""Failure detection on the device, through the C ABI.

The factorisation of Section 3 runs as one persistent launch whose clusters
wait on one another (reductions, pivot flags); every such wait is bounded and
reports GN_ETIMEOUT.  Non-finite inputs (x, a coefficient, an entry of
[A b]) are reported as GN_ENONFINITE and leave x alone.

Every failure is made on the host, none by faulting the GPU: a wait bound of
a few hundred cycles, which no message between the CTAs of a cluster can
meet, and NaN or infinite values written into the inputs.  After each failure
the same call with sound settings must succeed, which shows that the device
was left usable.
"""

import dataclasses
import time

import numpy as np
import pytest

import oracle
from paper_1402_2626_gb300 import inputs
from tests._util import PARITY_TOL, limb_diff, lstsq_sensitivity, term_scales

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GN_OK, GN_ENONFINITE, GN_ETIMEOUT = 0, 6, 7
PRECS = [("d", 1), ("dd", 2), ("qd", 4)]
SHORT_WAIT = 200  # SM cycles: far below one distributed-shared-memory round trip


def _gn():
    from paper_1402_2626_gb300 import build, gn

    build.build()
    return gn


def _matrix(m, ncols, L, seed):
    rng = np.random.default_rng(seed)
    A = np.zeros((m, ncols, 2, L))
    A[..., 0, 0] = rng.standard_normal((m, ncols))
    A[..., 1, 0] = rng.standard_normal((m, ncols))
    return A


@pytest.mark.parametrize("prec,L", PRECS)
def test_mgs_wait_timeout_then_recovers(prec, L):
    """A wait bound no reduction can meet: gn_mgs reports GN_ETIMEOUT promptly;
    with the default bound restored the same factorisation succeeds and
    matches the oracle."""
    gn = _gn()
    m = n = 256
    A = _matrix(m, n + 1, L, 11)
    s = gn.System(inputs.random_system(n, n, 2, 1, 1, seed=0))
    Ab = torch.tensor(np.ascontiguousarray(A.transpose(1, 0, 2, 3)), device="cuda")
    R = torch.zeros((n + 1, n + 1, 2, L), dtype=torch.float64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    prev = gn.set_wait_limit(SHORT_WAIT)
    try:
        assert prev > 0
        t0 = time.perf_counter()
        s.mgs(prec, Ab, R, st)
        torch.cuda.synchronize()
        elapsed = time.perf_counter() - t0
    finally:
        assert gn.set_wait_limit(0) == SHORT_WAIT
    assert int(st.item()) == GN_ETIMEOUT
    assert elapsed < 5.0  # every other wait gave up at once
    Ab.copy_(torch.tensor(np.ascontiguousarray(A.transpose(1, 0, 2, 3))))
    s.mgs(prec, Ab, R, st)
    torch.cuda.synchronize()
    assert int(st.item()) == GN_OK
    Qo, Ro = oracle.mgs(A, L, nthreads=8)
    Rg = R.cpu().numpy().transpose(1, 0, 2, 3)
    Qg = Ab.cpu().numpy().transpose(1, 0, 2, 3)
    # within the first-order perturbation bounds of this case (tests._util)
    kappa, cn, _ = lstsq_sensitivity(A, Ro)
    assert np.all(limb_diff(Rg, Ro) <= PARITY_TOL[L] * kappa * cn[None, :])
    assert np.all(limb_diff(Qg[:, :n], Qo[:, :n]) <= PARITY_TOL[L] * kappa)
    s.close()


def test_newton_wait_timeout_leaves_x():
    """The captured Newton step reads the bound when it runs: with the short
    bound gn_newton returns GN_ETIMEOUT, no step is applied and x is
    unchanged; with the default bound restored the step equals the oracle's."""
    gn = _gn()
    L = 2
    s = inputs.workload("gn32")
    sy = gn.System(s)
    x = torch.tensor(s.point("x0", L), device="cuda")
    sy.newton("dd", x, 1)  # captures the step graph with the default bound
    x.copy_(torch.tensor(s.point("x0", L)))
    gn.set_wait_limit(SHORT_WAIT)
    try:
        rep = sy.newton("dd", x, 3, raise_on_error=False)
    finally:
        gn.set_wait_limit(0)
    assert rep["status"] == GN_ETIMEOUT and rep["steps_done"] == 0
    assert np.array_equal(x.cpu().numpy(), s.point("x0", L))
    rep = sy.newton("dd", x, 1)
    assert rep["status"] == GN_OK
    xo, _, _, _ = oracle.newton_step(s, s.point("x0", L), L, nthreads=8)
    assert np.all(limb_diff(x.cpu().numpy(), xo) <= PARITY_TOL[L])
    sy.close()


def _with_bad_coef(system, value):
    """The system with the leading real limb of one coefficient replaced:
    the first term of polynomial 3 that has a variable."""
    t = next(t for t in range(int(system.poly_ptr[3]), int(system.poly_ptr[4]))
             if system.mono_ptr[t + 1] > system.mono_ptr[t])
    coef = system.coef.copy()
    coef[t, 0, 0] = value
    return dataclasses.replace(system, coef=coef), t


@pytest.mark.parametrize("arith", ["auto", "int", "fp64"])
@pytest.mark.parametrize("prec,L", PRECS)
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_newton_nonfinite_coefficient(prec, L, arith, bad):
    """A NaN or infinite coefficient, loaded through gn_system_create: every
    arithmetic reports GN_ENONFINITE from the first step and leaves x as it was."""
    gn = _gn()
    base = inputs.random_system(24, 20, (6, 12), (1, 6), 3, seed=901)
    s, _ = _with_bad_coef(base, bad)
    sy = gn.System(s, arith=arith)
    x = torch.tensor(s.point("x0", L), device="cuda")
    rep = sy.newton(prec, x, 2, raise_on_error=False)
    assert rep["status"] == GN_ENONFINITE and rep["steps_done"] == 0, rep
    assert np.array_equal(x.cpu().numpy(), s.point("x0", L))
    sy.close()


@pytest.mark.parametrize("prec,L", PRECS)
def test_set_coef_nonfinite_then_restore(prec, L):
    """A NaN placed by gn_system_set_coef is reported on the next step; the
    finite coefficients set back give the oracle's step again."""
    gn = _gn()
    s = inputs.random_system(24, 20, (6, 12), (1, 6), 3, seed=902)
    sy = gn.System(s)
    bad, _ = _with_bad_coef(s, np.nan)
    sy.set_coef(torch.tensor(bad.coef[:, :, :L], device="cuda"))
    x = torch.tensor(s.point("x0", L), device="cuda")
    rep = sy.newton(prec, x, 1, raise_on_error=False)
    assert rep["status"] == GN_ENONFINITE and rep["steps_done"] == 0
    assert np.array_equal(x.cpu().numpy(), s.point("x0", L))
    good = s.coef.copy()
    good[:, :, L:] = 0.0
    sy.set_coef(torch.tensor(good[:, :, :L], device="cuda"))
    rep = sy.newton(prec, x, 1)
    assert rep["status"] == GN_OK
    xo, _, _, _ = oracle.newton_step(dataclasses.replace(s, coef=good), s.point("x0", L), L)
    assert np.all(limb_diff(x.cpu().numpy(), xo) <= PARITY_TOL[L])
    sy.close()


@pytest.mark.parametrize("arith", ["auto", "fp64"])
@pytest.mark.parametrize("prec,L", PRECS)
def test_newton_nonfinite_start(prec, L, arith):
    gn = _gn()
    s = inputs.random_system(24, 20, (6, 12), (1, 6), 3, seed=903)
    sy = gn.System(s, arith=arith)
    x0 = s.point("x0", L)
    x0[5, 1, 0] = np.nan
    x = torch.tensor(x0, device="cuda")
    rep = sy.newton(prec, x, 1, raise_on_error=False)
    assert rep["status"] == GN_ENONFINITE and rep["steps_done"] == 0
    sy.close()


@pytest.mark.parametrize("arith", ["int", "fp64"])
@pytest.mark.parametrize("prec,L", PRECS)
def test_eval_nonfinite_coefficient_reaches_f_and_J(prec, L, arith):
    """gn_eval propagates a NaN coefficient as floating point would: f of its
    polynomial and the Jacobian entries of its variables turn NaN, every
    other entry matches the oracle's evaluation of the sound system."""
    gn = _gn()
    s = inputs.random_system(24, 20, (6, 12), (1, 6), 3, seed=904)
    bad, t = _with_bad_coef(s, np.nan)
    sy = gn.System(bad, arith=arith)
    x = torch.tensor(s.point("x0", L), device="cuda")
    f = torch.zeros((s.N, 2, L), dtype=torch.float64, device="cuda")
    J = torch.zeros((s.n, s.N, 2, L), dtype=torch.float64, device="cuda")
    sy.eval(prec, x, f, J)
    fh = f.cpu().numpy()
    Jh = J.cpu().numpy().transpose(1, 0, 2, 3)
    vs = set(int(v) for v in s.var[s.mono_ptr[t]:s.mono_ptr[t + 1]])
    assert np.isnan(fh[3]).any()
    for v in vs:
        assert np.isnan(Jh[3, v]).any()
    fo, Jo, _ = oracle.evaluate(s, s.point("x0", L), L)
    ok_rows = [i for i in range(s.N) if i != 3]
    assert np.all(np.isfinite(fh[ok_rows])) and np.all(np.isfinite(Jh[ok_rows]))
    Sf, SJ = term_scales(s, s.point("x0", L))
    assert np.all(limb_diff(fh[ok_rows], fo[ok_rows]) <= PARITY_TOL[L] * Sf[ok_rows])
    assert np.all(limb_diff(Jh[ok_rows], Jo[ok_rows]) <= PARITY_TOL[L] * SJ[ok_rows])
    sy.close()


@pytest.mark.parametrize("arith", ["int", "fp64"])
@pytest.mark.parametrize("prec,L", PRECS)
def test_lstsq_and_mgs_nonfinite(prec, L, arith):
    gn = _gn()
    m, n = 40, 33
    A = _matrix(m, n + 1, L, 12)
    A[17, 9, 1, 0] = np.inf
    s = gn.System(inputs.random_system(n, n, 2, 1, 1, seed=0), arith=arith)
    Ab = torch.tensor(np.ascontiguousarray(A.transpose(1, 0, 2, 3)), device="cuda")
    R = torch.zeros((n + 1, n + 1, 2, L), dtype=torch.float64, device="cuda")
    dx = torch.zeros((n, 2, L), dtype=torch.float64, device="cuda")
    with pytest.raises(gn.GnError) as e:
        s.lstsq(prec, Ab, R, dx)
    assert e.value.status == GN_ENONFINITE
    A[17, 9, 1, 0] = np.nan
    Ab.copy_(torch.tensor(np.ascontiguousarray(A.transpose(1, 0, 2, 3))))
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    s.mgs(prec, Ab, R, st)
    torch.cuda.synchronize()
    assert int(st.item()) == GN_ENONFINITE
    s.close()


def test_batch_nonfinite_system_reports_alone():
    """A NaN coefficient in one system of a batch: that system gets
    GN_ENONFINITE and keeps its x; the others advance to their roots."""
    gn = _gn()
    b = inputs.random_batch(6, 778, n_range=(16, 24))
    s_bad = 4
    p0 = int(b.sys_poly[s_bad])
    b.coef[int(b.poly_ptr[p0 + 1]), 1, 0] = np.nan
    L = 2
    g = gn.Batch(b)
    x = torch.tensor(b.point("x0", L), device="cuda")
    status = torch.zeros((b.S,), dtype=torch.int32, device="cuda")
    g.newton("dd", x, 2, status)
    torch.cuda.synchronize()
    st = status.cpu().numpy()
    xh = x.cpu().numpy()
    assert st[s_bad] == GN_ENONFINITE
    v0, v1 = int(b.sys_var[s_bad]), int(b.sys_var[s_bad + 1])
    assert np.array_equal(xh[v0:v1], b.point("x0", L)[v0:v1])
    for s in range(b.S):
        if s == s_bad:
            continue
        assert st[s] == GN_OK
        v0, v1 = int(b.sys_var[s]), int(b.sys_var[s + 1])
        d = xh[v0:v1].copy()
        d[:, :, 0] -= b.xstar[v0:v1]
        assert limb_diff(d, np.zeros_like(d)).max() < 1e-14  # two steps from 1e-6
    g.close()
