"""Plant plausible mistakes in copies of the oracle and check that the pins catch each.

Every mutant is a textual edit of ``oracle/gemm_oracle.c`` compiled into a temporary
library; the committed oracle itself is never modified.  A mutant passes only if it makes
at least one pin in ``tests/oracle_pins.py`` fail."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from tests import oracle_pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "gemm_oracle.c")

MUTANTS = {
    "dropped_beta_term": ("if (beta != 0.0) t = t + beta * c[i];",
                          "if (beta != 0.0) t = t + 0.0 * c[i];"),
    "beta_zero_reads_C": ("if (beta != 0.0) t = t + beta * c[i];", "t = t + beta * c[i];"),
    "dropped_alpha": ("t = alpha * s[i];", "t = s[i];"),
    "wrong_sign": ("s[i] = s[i] + prod;", "s[i] = s[i] - prod;"),
    "transposed_A": ("return a_notrans ? A[i + p * lda] : A[p + i * lda];",
                     "return a_notrans ? A[p + i * lda] : A[i + p * lda];"),
    "transposed_B": ("return b_notrans ? B[p + j * ldb] : B[j + p * ldb];",
                     "return b_notrans ? B[j + p * ldb] : B[p + j * ldb];"),
    "ldc_as_m": ("double *c = C + j * ldc;", "double *c = C + j * m;"),
    "lda_off_by_one": ("return a_notrans ? A[i + p * lda] : A[p + i * lda];",
                       "return a_notrans ? A[i + p * (lda - 1)] : A[p + i * lda];"),
    "last_k_dropped": ("for (int64_t p = 0; p < k; ++p) {\n                        double b",
                       "for (int64_t p = 0; p + 1 < k; ++p) {\n                        double b"),
    "ldc_check_off": ("if (ldc < (m > 1 ? m : 1)) return -13;", ""),
    "fp32_accumulator": ("double prod = op_a(A, lda, a_notrans, i, p) * b;\n"
                         "                            s[i] = s[i] + prod;",
                         "float prod = (float)(op_a(A, lda, a_notrans, i, p) * b);\n"
                         "                            s[i] = (float)(s[i] + prod);"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = src.replace(old, new, 1)
    cpath = tmp_path / f"{name}.c"
    cpath.write_text(mutated)
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-std=c99", "-shared",
                    "-fPIC", str(cpath), "-o", str(so), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    i64, dbl, ptr = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    lib.oracle_gemm.argtypes = [ctypes.c_char, ctypes.c_char, i64, i64, i64, dbl, ptr, i64,
                                ptr, i64, dbl, ptr, i64, ctypes.c_int]
    lib.oracle_gemm.restype = ctypes.c_int

    def gemm(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, nthreads=1):
        def p(a):
            return a.ctypes.data_as(ctypes.c_void_p)
        return lib.oracle_gemm(ta.encode(), tb.encode(), m, n, k, float(alpha), p(A), lda,
                               p(B), ldb, float(beta), p(C), ldc, nthreads)
    return gemm


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    gemm = _build_mutant(tmp_path, name, old, new)
    caught = []
    for pin in oracle_pins.ALL_PINS:
        try:
            with np.errstate(all="ignore"):
                pin(gemm)
        except (AssertionError, ValueError, IndexError) as e:  # noqa: PERF203
            caught.append(pin.__name__)
            break
    assert caught, f"mutant {name} passed every pin"
