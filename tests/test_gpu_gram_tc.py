"""The Gram matrix of the mixed-precision solver's CholeskyQR on the tensor
cores (BF16 digit-plane products in tensor memory, combined in 128-bit
integers) against an exact CPU reference and against the integer-pipe form.

Section 5.2 of the paper points to double-precision methods for the linear
solve; CholeskyQR's Gram matrix G = [A b]^H [A b] is its O(m n^2) part.  The
driver tests/native/gram_check.cu is built from the library's object files,
so it calls the kernels below the C ABI: for integer entries times
power-of-two column scales the exact G (128-bit integer sums on the CPU) is
a matrix of doubles that both GPU forms must reproduce bit for bit; for
Gaussian entries the two forms, each exact for the columns rounded to 56 and
62 bits and then rounded once, must agree to 2^-51 of ||a_i|| ||a_j||.  The
end-to-end parity of the solver that uses it is in test_gpu_mixed.
"""

import json
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_gram_tensor_cores_exact(tmp_path):
    from paper_1402_2626_gb300 import build

    build.build()
    objs = sorted(os.path.join(build.BUILD, f) for f in os.listdir(build.BUILD) if f.endswith(".o"))
    exe = str(tmp_path / "gram_check")
    subprocess.run([build.nvcc(), *build.ARCH, "-O2", "-std=c++17", os.path.join(HERE, "native", "gram_check.cu"),
                    *objs, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    lines = [json.loads(l) for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 6, out.stdout + out.stderr
    for c in lines:
        assert c["ok"] == 1, c
        assert c["cuda"] == 0 and c["status"] == 0, c
        if c["integer"]:
            assert c["exact_tc"] == c["checked"] and c["differ"] == 0, c
    assert out.returncode == 0
