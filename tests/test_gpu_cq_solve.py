"""The triangular solves of the mixed-precision solver's CholeskyQR (the
float-float factor's diagonal-block inverses and the blocked solves on one
8-CTA cluster) against substitution in double on the CPU.

The Gauss-Newton step of Section 4 solves R dx = y with the factor of
[J, -f] (Section 3, eq. 5); the refinement solves R^H w = J^H b, then
R dx = w.  The driver tests/native/cq_solve_check.cu is built from the
library's object files, so it calls the kernels below the C ABI with factors
of known values: one block, ragged last blocks, CTAs owning several blocks,
the largest size, and right-hand sides far below the float range.  The
end-to-end parity of the solver that uses them is in test_gpu_mixed.
"""

import json
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_cq_solves_against_cpu(tmp_path):
    from paper_1402_2626_gb300 import build

    build.build()
    objs = sorted(os.path.join(build.BUILD, f) for f in os.listdir(build.BUILD) if f.endswith(".o"))
    exe = str(tmp_path / "cq_solve_check")
    subprocess.run([build.nvcc(), *build.ARCH, "-O2", "-std=c++17",
                    os.path.join(HERE, "native", "cq_solve_check.cu"), *objs, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    lines = [json.loads(l) for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 8, out.stdout + out.stderr
    for c in lines:
        assert c["cuda"] == 0 and c["launch"] == 0 and c["status"] == 0, c
        assert c["rel_err"] <= 2.0 ** -40, c
        assert c["ok"] == 1, c
    assert out.returncode == 0
