"""GPU parity of mixed-precision Gauss-Newton (double factorisation, DD or QD
residuals, gn_newton_mixed) against the CPU oracle, through the C ABI."""

import numpy as np
import pytest

import oracle
from paper_1402_2626_gb300 import inputs
from tests._util import ORACLE_OP_BOUND, PARITY_TOL, limb_diff, term_scales

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    # 32 unknowns: CholeskyQR with the Gram matrix on the tensor cores
    ("overdetermined", dict(N=48, n=32, M=(8, 16), k=(1, 6), dmax=4, seed=601)),
    # below 32 unknowns: the integer MGS double step
    ("square", dict(N=24, n=24, M=(8, 24), k=(1, 5), dmax=3, seed=602)),
    # above 2048 rows: CholeskyQR with the Gram matrix on the integer pipe
    ("tall", dict(N=2100, n=32, M=(3, 6), k=(1, 4), dmax=3, seed=603)),
    # three Cholesky panels (the lookahead) and three solve blocks, the last
    # one ragged (77 = 2 x 32 + 13)
    ("ragged", dict(N=120, n=77, M=(4, 10), k=(1, 5), dmax=3, seed=604)),
]


def _gn():
    from paper_1402_2626_gb300 import build, gn

    build.build()
    return gn


def _err_vs_root(s, x):
    d = np.array(x, dtype=np.float64, copy=True)
    d[:, :, 0] -= s.xstar
    return float(limb_diff(d, np.zeros_like(d)).max())


@pytest.mark.parametrize("arith", ["auto", "fp64"])
@pytest.mark.parametrize("prec,L,refine", [("dd", 2, 3), ("qd", 4, 6)])
@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
def test_mixed_parity_small(name, kw, prec, L, refine, arith):
    gn = _gn()
    s = inputs.random_system(kw["N"], kw["n"], kw["M"], kw["k"], kw["dmax"], seed=kw["seed"])
    sy = gn.System(s, arith=arith)
    x = torch.tensor(s.point("x0", L), device="cuda")
    rep = sy.newton_mixed(prec, x, 3, refine)
    xh = x.cpu().numpy()
    xo, ho = oracle.newton_mixed(s, s.point("x0", L), L, 3, refine)
    assert limb_diff(xh, xo).max() <= PARITY_TOL[L]
    assert _err_vs_root(s, xh) <= PARITY_TOL[L]
    assert rep["steps_done"] == 3 + refine
    # the double phase is plain double Gauss-Newton: same norms as the oracle's
    for k in range(3):
        assert rep["res_norm"][k] == pytest.approx(ho[k][0], rel=1e-6, abs=1e-14)
    # refinement: each ||dx|| shrinks by 1e8 or lands at the rounding floor
    # of precision L (about u_L ||x||)
    dx = rep["dx_norm"][3:]
    floor = 100 * ORACLE_OP_BOUND[L] * np.sqrt(s.n)
    for a, b in zip(dx, dx[1:]):
        assert b <= max(1e-8 * a, floor), dx
    sy.close()


def test_mixed_tol_stops_early():
    gn = _gn()
    _, kw = CASES[0]
    s = inputs.random_system(kw["N"], kw["n"], kw["M"], kw["k"], kw["dmax"], seed=kw["seed"])
    sy = gn.System(s)
    x = torch.tensor(s.point("x0", 4), device="cuda")
    rep = sy.newton_mixed("qd", x, 3, 20, tol=1e-40)
    assert rep["status"] == 0 and 3 + 2 <= rep["steps_done"] < 3 + 20
    assert rep["dx_norm"][-1] <= 1e-40 * np.sqrt(s.n)
    # an unreachable tolerance: every step taken, GN_ENOCONV
    x = torch.tensor(s.point("x0", 4), device="cuda")
    rep = sy.newton_mixed("qd", x, 3, 2, tol=1e-300, raise_on_error=False)
    assert rep["status"] == 5 and rep["steps_done"] == 5
    sy.close()


def test_mixed_full_size_qd():
    """The mixed-precision workload at full size (N = 1536, n = 1024, 63 terms
    of 8 variables plus a constant per polynomial, exponents 1..4): three
    double steps and five QD refinement steps reach the exact root at QD
    accuracy; residuals of sampled rows, evaluated by the oracle in QD at the
    GPU's x, are at the QD rounding level of their terms."""
    gn = _gn()
    s = inputs.workload("mix1536")
    sy = gn.System(s)
    x = torch.tensor(s.point("x0", 4), device="cuda")
    rep = sy.newton_mixed("qd", x, 3, 5)
    xh = x.cpu().numpy()
    assert _err_vs_root(s, xh) <= PARITY_TOL[4]
    for rows in ((0, 24), (700, 724), (1512, 1536)):
        f, _, _ = oracle.evaluate(s, xh, 4, rows=rows, jacobian=False, nthreads=8)
        Sf, _ = term_scales(s, xh, rows=rows)
        assert np.all(limb_diff(f, np.zeros_like(f)) <= PARITY_TOL[4] * Sf)
    assert rep["steps_done"] == 8
    sy.close()
