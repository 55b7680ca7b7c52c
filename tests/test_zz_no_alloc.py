"""gn_eval_noalloc: evaluation for callers that cannot allocate device memory
when they evaluate (inside someone else's stream capture, in a loop where
allocator calls are forbidden, or with device memory handed out by a fixed
pool).  It uses the library's one static scratch array instead of a workspace.

Checked through the C ABI against gn_eval on two calls in a row (the second
finds the scratch holding the first call's contents), that the call does not
change the device's free memory, and that a system too large for the scratch
is rejected with GN_EINVAL.  This file is collected last on purpose.
"""

import numpy as np
import pytest

from paper_1402_2626_gb300 import inputs
from tests._util import PARITY_TOL, limb_diff

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = [("d", 1), ("dd", 2), ("qd", 4)]


def _gn():
    from paper_1402_2626_gb300 import build, gn

    build.build()
    return gn


def _buffers(system, L):
    f = torch.full((system.N, 2, L), np.nan, dtype=torch.float64, device="cuda")
    J = torch.full((system.n, system.N, 2, L), np.nan, dtype=torch.float64, device="cuda")
    return f, J


@pytest.mark.parametrize("prec,L", PRECS)
def test_noalloc_matches_gn_eval_twice(prec, L):
    gn = _gn()
    for system in (inputs.workload("gn32"), inputs.random_system(37, 29, (20, 45), (1, 14), 5, seed=77)):
        s = gn.System(system, arith="fp64")  # the arithmetic gn_eval_noalloc uses
        x = torch.tensor(system.point("x0", L), device="cuda")
        f_ref, J_ref = _buffers(system, L)
        s.eval(prec, x, f_ref, J_ref)
        for _ in range(2):  # the second call reuses scratch left by the first
            f, J = _buffers(system, L)
            s.eval_noalloc(prec, x, f, J)
            torch.cuda.synchronize()
            tol = PARITY_TOL[L]
            assert np.all(limb_diff(f.cpu().numpy(), f_ref.cpu().numpy()) <= tol)
            assert np.all(limb_diff(J.cpu().numpy(), J_ref.cpu().numpy()) <= tol)
        s.close()


@pytest.mark.parametrize("warm_prec,warm_L", [("dd", 2), ("d", 1)])
def test_noalloc_allocates_nothing(warm_prec, warm_L):
    """After one first call in one precision, calls in every precision leave
    the device's free memory unchanged (the first call also loads the code of
    the other precisions' kernels)."""
    gn = _gn()
    warm = inputs.random_system(4, 4, 4, (1, 3), 3, seed=1)
    w = gn.System(warm)
    xw = torch.tensor(warm.point("x0", warm_L), device="cuda")
    w.eval_noalloc(warm_prec, xw)  # first call on the device: looks up the scratch
    torch.cuda.synchronize()
    system = inputs.workload("gn32")
    s = gn.System(system)  # loading the system allocates; evaluating must not
    bufs = {}
    for prec, L in PRECS:
        x = torch.tensor(system.point("x0", L), device="cuda")
        bufs[prec] = (x, *_buffers(system, L))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        for prec, _L in PRECS:
            x, f, J = bufs[prec]
            s.eval_noalloc(prec, x, f, J)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for prec, _L in PRECS:
        assert not torch.isnan(bufs[prec][2]).any()
    s.close()
    w.close()


def test_noalloc_full_size_and_limit():
    gn = _gn()
    system = inputs.workload("gn256")  # 65,792 terms, 1,048,576 occurrences
    s = gn.System(system, arith="fp64")  # the arithmetic gn_eval_noalloc uses
    x = torch.tensor(system.point("x0", 2), device="cuda")
    f_ref, J_ref = _buffers(system, 2)
    s.eval("dd", x, f_ref, J_ref)
    f, J = _buffers(system, 2)
    s.eval_noalloc("dd", x, f, J)
    torch.cuda.synchronize()
    assert np.all(limb_diff(f.cpu().numpy(), f_ref.cpu().numpy()) <= PARITY_TOL[2])
    assert np.all(limb_diff(J.cpu().numpy(), J_ref.cpu().numpy()) <= PARITY_TOL[2])
    # quad double needs 64 B per occurrence: over the 64 MiB scratch
    x4 = torch.tensor(system.point("x0", 4), device="cuda")
    f4, J4 = _buffers(system, 4)
    with pytest.raises(gn.GnError) as e:
        s.eval_noalloc("qd", x4, f4, J4)
    assert e.value.status == 1
    s.close()
