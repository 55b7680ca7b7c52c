"""GPU parity of batched Gauss-Newton (many independent systems per launch)
against the CPU oracle, system by system, through the C ABI."""

import numpy as np
import pytest

import oracle
from paper_1402_2626_gb300 import inputs
from tests._util import PARITY_TOL, limb_diff

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = [("d", 1), ("dd", 2), ("qd", 4)]


def _gn():
    from paper_1402_2626_gb300 import build, gn

    build.build()
    return gn


def run_batch(b, L, prec, steps):
    gn = _gn()
    g = gn.Batch(b)
    x = torch.tensor(b.point("x0", L), device="cuda")
    status = torch.zeros((b.S,), dtype=torch.int32, device="cuda")
    norms = torch.zeros((steps, b.S, 2), dtype=torch.float64, device="cuda")
    g.newton(prec, x, steps, status, norms)
    torch.cuda.synchronize()
    out = x.cpu().numpy(), status.cpu().numpy(), norms.cpu().numpy()
    g.close()
    return out


@pytest.mark.parametrize("prec,L", PRECS)
def test_batch_one_step_parity(prec, L):
    """One step on every system of a small batch (n in [16, 40]) against the
    oracle's step on that system alone."""
    b = inputs.random_batch(12, 31337, n_range=(16, 40))
    x, st, norms = run_batch(b, L, prec, 1)
    assert not st.any(), st
    for s in range(b.S):
        sy = b.system(s)
        v0, v1 = int(b.sys_var[s]), int(b.sys_var[s + 1])
        xo, _, fo, _ = oracle.newton_step(sy, sy.point("x0", L), L, nthreads=8)
        assert np.all(limb_diff(x[v0:v1], xo) <= PARITY_TOL[L]), (s, float(limb_diff(x[v0:v1], xo).max()))
        fn = float(np.sqrt((fo[:, :, 0] ** 2).sum()))
        assert norms[0, s, 0] == pytest.approx(fn, rel=1e-9)


@pytest.mark.parametrize("prec,L", [("d", 1), ("dd", 2)])
def test_batch_converges(prec, L):
    """Property over a batch of mixed sizes (n in [16, 128]): quadratic
    convergence of every system to its built-in root."""
    b = inputs.random_batch(48, 4242, n_range=(16, 128))
    x, st, norms = run_batch(b, L, prec, 4)
    assert not st.any(), st
    d = x.copy()
    d[:, :, 0] -= b.xstar
    err = limb_diff(d, np.zeros_like(d))
    assert err.max() <= PARITY_TOL[L], float(err.max())
    # ||dx|| contracts quadratically: ||dx_1|| <= C ||dx_0||^2
    assert np.all(norms[0, :, 1] < 1e-4)
    assert np.all(norms[1, :, 1] <= 1e3 * norms[0, :, 1] ** 2)


def test_batch_singular_system_reports_alone():
    """A system whose Jacobian loses rank gets GN_ESINGULAR; the others advance."""
    b = inputs.random_batch(6, 777, n_range=(16, 24))
    s_bad = 2
    # zero the coefficient of every term of system s_bad that contains its
    # variable 0: the structure stays valid, Jacobian column 0 vanishes
    p0, p1 = int(b.sys_poly[s_bad]), int(b.sys_poly[s_bad + 1])
    t0, t1 = int(b.poly_ptr[p0]), int(b.poly_ptr[p1])
    for t in range(t0, t1):
        a, c = int(b.mono_ptr[t]), int(b.mono_ptr[t + 1])
        if np.any(b.var[a:c] == 0):
            b.coef[t] = 0.0
    x, st, norms = run_batch(b, 2, "dd", 2)
    assert st[s_bad] == 4
    ok = [s for s in range(b.S) if s != s_bad]
    assert not st[ok].any()
    for s in ok:
        v0, v1 = int(b.sys_var[s]), int(b.sys_var[s + 1])
        d = x[v0:v1].copy()
        d[:, :, 0] -= b.xstar[v0:v1]
        assert limb_diff(d, np.zeros_like(d)).max() < 1e-14  # two steps from 1e-6


def test_batch_full_size_sampled():
    """The batched configuration at full size (4096 systems, n in [16, 128],
    complex DD): sampled systems match the oracle's first step one by one;
    three more steps bring every system to its root at DD accuracy."""
    gn = _gn()
    b = inputs.batch_workload("batch4096")
    L = 2
    g = gn.Batch(b)
    x = torch.tensor(b.point("x0", L), device="cuda")
    status = torch.zeros((b.S,), dtype=torch.int32, device="cuda")
    g.newton("dd", x, 1, status)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    assert not status.cpu().numpy().any()
    order = np.argsort(-b.n, kind="stable")
    for s in (int(order[0]), int(order[-1]), 2024):  # the largest, the smallest, one more
        sy = b.system(s)
        v0, v1 = int(b.sys_var[s]), int(b.sys_var[s + 1])
        xo, _, _, _ = oracle.newton_step(sy, sy.point("x0", L), L, nthreads=16)
        assert np.all(limb_diff(xh[v0:v1], xo) <= PARITY_TOL[L]), s
    g.newton("dd", x, 3, status)
    torch.cuda.synchronize()
    assert not status.cpu().numpy().any()
    d = x.cpu().numpy()
    d[:, :, 0] -= b.xstar
    assert limb_diff(d, np.zeros_like(d)).max() <= PARITY_TOL[L]
    # the tuner's choices are among its candidates
    tune = g.tuning("dd")
    assert tune["eval_block"] in (64, 128, 256) and tune["solve_threads"] in (128, 256)
    assert tune["eval_lanes"] in (1, 2)
    assert tune["solve_grid"] % torch.cuda.get_device_properties(0).multi_processor_count == 0
    with pytest.raises(gn.GnError):
        g.tuning("qd")  # never stepped in QD
    g.close()
