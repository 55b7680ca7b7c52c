"""How the least-squares solver (Section 3) behaves away from well-scaled
inputs, through the C ABI.

Column scaling: modified Gram-Schmidt commutes with a diagonal scaling of
the columns by powers of two (Q unchanged, column j of R times 2^e_j).  The
integer form keeps one exponent per column and the FP64 form scales every
operation exactly, so both must reproduce that bit for bit.

Row scaling: rows of very different magnitude make [A b] ill-conditioned;
the GPU keeps K-limb mantissas at one exponent per column, the oracle L-limb
cascades per entry.  Their results must still agree within the first-order
perturbation bounds of the scaled problem (tests._util.lstsq_sensitivity)
with the stated tolerance, for scalings up to 2^±20 between rows (kappa of
6e5 and 4e10 here, which the double-precision SVD of the oracle's R still
resolves).
"""

import numpy as np
import pytest

import oracle
from paper_1402_2626_gb300 import inputs
from tests._util import PARITY_TOL, limb_diff, lstsq_sensitivity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = [("d", 1), ("dd", 2), ("qd", 4)]


def _gn():
    from paper_1402_2626_gb300 import build, gn

    build.build()
    return gn


def _matrix(m, ncols, L, seed):
    rng = np.random.default_rng(seed)
    A = np.zeros((m, ncols, 2, L))
    A[..., 0, 0] = rng.standard_normal((m, ncols))
    A[..., 1, 0] = rng.standard_normal((m, ncols))
    if L > 1:
        A[..., :, 1] = A[..., :, 0] * 2.0 ** -55 * rng.standard_normal((m, ncols, 2))
    return A


def _lstsq(gn, s, A, L, prec):
    m, ncols = A.shape[0], A.shape[1]
    Ab = torch.tensor(np.ascontiguousarray(A.transpose(1, 0, 2, 3)), device="cuda")
    R = torch.zeros((ncols, ncols, 2, L), dtype=torch.float64, device="cuda")
    dx = torch.zeros((ncols - 1, 2, L), dtype=torch.float64, device="cuda")
    s.lstsq(prec, Ab, R, dx)
    torch.cuda.synchronize()
    return (Ab.cpu().numpy().transpose(1, 0, 2, 3), R.cpu().numpy().transpose(1, 0, 2, 3),
            dx.cpu().numpy())


@pytest.mark.parametrize("arith", ["int", "fp64"])
@pytest.mark.parametrize("prec,L", PRECS)
def test_column_scaling_is_exact(prec, L, arith):
    gn = _gn()
    m, n = 150, 120
    A = _matrix(m, n + 1, L, 31)
    e = np.random.default_rng(32).integers(-60, 61, size=n + 1)
    As = A * np.ldexp(1.0, e)[None, :, None, None]
    s = gn.System(inputs.random_system(n, n, 2, 1, 1, seed=0), arith=arith)
    Q, R, _ = _lstsq(gn, s, A, L, prec)
    Qs, Rs, _ = _lstsq(gn, s, As, L, prec)
    s.close()
    assert np.array_equal(Qs[:, :n], Q[:, :n])
    assert np.array_equal(Rs, R * np.ldexp(1.0, e)[None, :, None, None])


@pytest.mark.parametrize("prec,L", PRECS)
@pytest.mark.parametrize("spread", [10, 20])
def test_row_scaling_within_bounds(prec, L, spread):
    gn = _gn()
    m, n = 96, 80
    A = _matrix(m, n + 1, L, 40 + spread)
    rows = np.random.default_rng(41).integers(-spread, spread + 1, size=m)
    A = A * np.ldexp(1.0, rows)[:, None, None, None]
    s = gn.System(inputs.random_system(n, n, 2, 1, 1, seed=0))
    Q, R, dx = _lstsq(gn, s, A, L, prec)
    s.close()
    Qo, Ro = oracle.mgs(A, L, nthreads=8)
    dxo = oracle.backsub(Ro, L)
    tol = PARITY_TOL[L]
    kappa, cn, fx = lstsq_sensitivity(A, Ro)
    assert np.all(limb_diff(R, Ro) <= tol * kappa * cn[None, :]), kappa
    assert np.all(limb_diff(Q[:, :n], Qo[:, :n]) <= tol * kappa), kappa
    assert np.all(limb_diff(dx, dxo) <= tol * fx), kappa
