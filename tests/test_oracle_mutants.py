"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/oracle.c (on the CPU, in a
temporary directory), builds it, and runs the oracle pin tests against it in
a child process: at least one pin must fail.  The mistakes are the kinds the
pins are meant to catch: a dropped term, a wrong sign, a wrong index, a
transposed operand, a dropped limb.
"""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = [
    ("conjugation dropped in q^H a",
     "      x_grow_prod(&e, a[i], b[L + j]);\n      x_grow_prod(&e, -a[L + i], b[j]);",
     "      x_grow_prod(&e, a[i], b[L + j]);\n      x_grow_prod(&e, a[L + i], b[j]);"),
    ("sign of im*im in the complex product",
     "      x_grow_prod(&e, -a[L + i], b[L + j]);\n    }\n  x_round(&e, L, re);\n  x_init(&e);\n  for (int i = 0; i < L; i++)\n    for (int j = 0; j < L; j++) {\n      x_grow_prod(&e, a[i], b[L + j]);\n      x_grow_prod(&e, a[L + i], b[j]);",
     "      x_grow_prod(&e, a[L + i], b[L + j]);\n    }\n  x_round(&e, L, re);\n  x_init(&e);\n  for (int i = 0; i < L; i++)\n    for (int j = 0; j < L; j++) {\n      x_grow_prod(&e, a[i], b[L + j]);\n      x_grow_prod(&e, a[L + i], b[j]);"),
    ("exponent factor dropped on the last partial",
     "c_scale_int(L, tmp, d[k - 1], part + (int64_t)(k - 1) * W);",
     "c_scale_int(L, tmp, 1, part + (int64_t)(k - 1) * W);"),
    ("wrong variable in the backward product",
     "c_mul(L, B, xv(cx, v[s]), B);",
     "c_mul(L, B, xv(cx, v[s - 1]), B);"),
    ("common factor uses x^d instead of x^(d-1)",
     "const double *tv = pow_tab + ((int64_t)v[s] * pmax + (d[s] - 2)) * W;",
     "const double *tv = pow_tab + ((int64_t)v[s] * pmax + (d[s] - 1 < pmax ? d[s] - 1 : d[s] - 2)) * W;"),
    ("constant term dropped",
     "    memcpy(term, a, sizeof(double) * W);\n    return;",
     "    c_zero(L, term);\n    return;"),
    ("transposed R in back substitution",
     "c_mul(L, R + ((int64_t)j * ldr + l) * W, x + (int64_t)j * W, p);",
     "c_mul(L, R + ((int64_t)l * ldr + j) * W, x + (int64_t)j * W, p);"),
    ("pivot column not normalized",
     "for (int i = 0; i < m; i++) c_div_real(L, ak + i * W, rkk, ak + i * W);",
     "for (int i = 0; i < m && 0; i++) c_div_real(L, ak + i * W, rkk, ak + i * W);"),
    ("last limb dropped in rounding",
     "    out[l] = approx;\n    if (approx != 0.0) x_grow(e, -approx);",
     "    out[l] = (l == L - 1 && L > 1) ? 0.0 : approx;\n    if (approx != 0.0) x_grow(e, -approx);"),
    ("no conjugate in the forward substitution with R^H",
     "c_conj_mul(L, R + ((int64_t)l * ldr + j) * W, w + (int64_t)j * W, p);",
     "c_mul(L, R + ((int64_t)l * ldr + j) * W, w + (int64_t)j * W, p);"),
    ("R read untransposed in the forward substitution",
     "c_conj_mul(L, R + ((int64_t)l * ldr + j) * W, w + (int64_t)j * W, p);",
     "c_conj_mul(L, R + ((int64_t)j * ldr + l) * W, w + (int64_t)j * W, p);"),
    ("lambda conjugated instead of the monomial",
     "c_conj_mul(L, mono + t * W, lam + (int64_t)i * W, grad + t * W);",
     "c_conj_mul(L, lam + (int64_t)i * W, mono + t * W, grad + t * W);"),
    ("sign of the coefficient gradient",
     "for (int l = 0; l < W; l++) grad[t * W + l] = -grad[t * W + l];",
     "for (int l = 0; l < W; l++) grad[t * W + l] = grad[t * W + l];"),
    ("exponent ignored in the monomial values",
     "for (int r = 0; r < exp[o]; r++) c_mul(L, acc, x + (int64_t)var[o] * W, acc);",
     "for (int r = 0; r < 1; r++) c_mul(L, acc, x + (int64_t)var[o] * W, acc);"),
    ("projection added instead of subtracted in the MGS update",
     "        c_mul(L, r, ak + i * W, p);\n        c_sub(L, aj + i * W, p, aj + i * W);",
     "        c_mul(L, r, ak + i * W, p);\n        c_add(L, aj + i * W, p, aj + i * W);"),
    ("pivot norm as a^T a instead of a^H a",
     "      x_grow_prod(&e, a[L + i], a[L + j]);\n    }\n  x_round(&e, L, r);",
     "      x_grow_prod(&e, -a[L + i], a[L + j]);\n    }\n  x_round(&e, L, r);"),
    ("power table squares instead of multiplying by x",
     "        c_mul(L, pow_tab + ((int64_t)v * pmax + p - 2) * W, xv(&cx, v),",
     "        c_mul(L, pow_tab + ((int64_t)v * pmax + p - 2) * W, pow_tab + ((int64_t)v * pmax + p - 2) * W,"),
    ("update subtracts instead of adds",
     "for (int i = 0; i < n; i++) c_add(L, x + i * W, dx + i * W, x + i * W);",
     "for (int i = 0; i < n; i++) c_sub(L, x + i * W, dx + i * W, x + i * W);"),
]


@pytest.mark.slow
@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(name, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique/found: {name}"
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    "-o", str(so), str(mut), "-lm"], check=True)
    env = dict(os.environ, ORACLE_LIB_OVERRIDE=str(so))
    r = subprocess.run(
        [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
         "tests/test_oracle_arith.py", "tests/test_oracle_eval.py",
         "tests/test_oracle_mgs.py", "tests/test_oracle_newton.py",
         "tests/test_oracle_adjoint.py"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught the mutant: {name}\n{r.stdout[-2000:]}"
