"""Pins of the oracle's Gauss-Newton step (Section 4).

* One step equals the exact least-squares step of the normal equations
  (exact rationals) on a tiny overdetermined system.
* From x* + 1e-6 on the generated workloads the error contracts
  quadratically (e_{k+1} <= C e_k^2) down to the precision floor, as the
  paper reports for its benchmarks (Section 5: quadratic convergence from
  H = 1 on the Chandrasekhar system, full precision in a few steps on
  cyclic n-roots).
"""

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_1402_2626_gb300 import inputs
from tests._util import ORACLE_OP_BOUND, cdiff, cfr, term_scales

FLOOR = {1: 1e-13, 2: 1e-26, 4: 1e-58}


@pytest.mark.parametrize("L", [1, 2, 4])
def test_step_matches_exact_lstsq(L):
    s = inputs.random_system(5, 3, (3, 5), (1, 3), 3, seed=404)  # N > n
    x = s.point("x0", L)
    _, dx, f, _ = oracle.newton_step(s, x, L)
    dxe = exact.lstsq_step(s, x, L=L)
    scale = max(abs(exact.to_float(v)) for v in dxe)
    # f carries rounding errors ~ u_L * S_f; the step amplifies them by
    # about |dx| / |f| (the size of J's pseudo-inverse)
    Sf, _ = term_scales(s, x)
    fmax = float(np.abs(oracle.to_complex(f)).max())
    bound = ORACLE_OP_BOUND[L] * 1e3 * (scale / fmax) * float(Sf.max())
    for v in range(s.n):
        assert cdiff(cfr(dx[v]), dxe[v]) <= bound
        assert bound < 1e-6 * scale  # the pin is far tighter than the step itself


@pytest.mark.parametrize("L", [1, 2, 4])
def test_quadratic_convergence_gn32(L):
    s = inputs.workload("gn32")
    xs = s.xstar[:, 0] + 1j * s.xstar[:, 1]
    x = s.point("x0", L)
    errs = []
    for _ in range(4):
        x, dx, _, _ = oracle.newton_step(s, x, L)
        d = x.copy()
        d[:, 0, 0] -= s.xstar[:, 0]
        d[:, 1, 0] -= s.xstar[:, 1]
        errs.append(float(np.abs(d[:, 0].sum(-1) + 1j * d[:, 1].sum(-1)).max()))
    e0 = float(np.abs((s.x0[:, 0] + 1j * s.x0[:, 1]) - xs).max())
    prev = e0
    for e in errs:
        if prev > FLOOR[L] * 1e-3:
            assert e <= 1e4 * prev * prev + FLOOR[L] * 1e-2, (errs, e0)
        prev = e
    assert errs[-1] <= FLOOR[L]
