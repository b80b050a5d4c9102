"""Pins of the SYRK oracle (oracle/syrk_oracle.c) against what the definition and the
mathematics fix, independently of the oracle itself, and planted mistakes that must fail
them.  CPU only.

* exact rational brute force (fractions.Fraction) on tiny shapes, every uplo and trans;
* a hand-worked product (below), bit-exact;
* integer operands: exact against numpy's int64 product;
* the reduction to the (separately pinned) GEMM oracle: with B = A and the transposed
  operand order, every triangle entry is bit-identical, since both sum a(i,p) a(j,p) for p
  in increasing order from +0.0 and then form alpha*S + beta*C;
* reference-BLAS rules: argument codes, quick returns, beta == 0 never reads C,
  alpha == 0 never reads A, the other triangle and the ld gap never touched."""
import ctypes
import itertools
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2302_08417_gb300 import inputs

U = 2.0 ** -53
SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "syrk_oracle.c")


def _tri(uplo, n):
    """Boolean n x n mask of the referenced triangle."""
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return (i >= j) if uplo in "Ll" else (i <= j)


def _a(A, lda, trans, i, p):
    return A[i + p * lda] if trans in "Nn" else A[p + i * lda]


def pin_bruteforce(syrk):
    rng = np.random.Generator(np.random.PCG64(1))
    for uplo, trans, n, k, pad in itertools.product("LU", "NTc", (0, 1, 2, 3, 5), (0, 1, 2, 3),
                                                    (0, 3)):
        rows = n if trans in "Nn" else k
        cols = k if trans in "Nn" else n
        lda = max(1, rows + pad)
        ldc = max(1, n + pad)
        for alpha, beta in ((1.0, 0.0), (-0.5, 0.5), (2.0, 1.0), (0.0, -1.5)):
            A = inputs.colmajor(rng, rows, cols, lda)
            C0 = inputs.colmajor(rng, n, n, ldc)
            C = C0.copy()
            assert syrk(uplo, trans, n, k, alpha, A, lda, beta, C, ldc) == 0
            for i, j in itertools.product(range(n), range(n)):
                inside = (i >= j) if uplo == "L" else (i <= j)
                got, old = C[i + j * ldc], C0[i + j * ldc]
                if not inside:
                    assert got == old or (np.isnan(got) and np.isnan(old))
                    continue
                if (alpha == 0.0 or k == 0) and beta == 1.0:
                    assert got == old
                    continue
                s = sum((Fraction(_a(A, lda, trans, i, p)) * Fraction(_a(A, lda, trans, j, p))
                         for p in range(k)), Fraction(0))
                exact = Fraction(alpha) * s + (Fraction(beta) * Fraction(old) if beta else 0)
                mag = sum((abs(Fraction(_a(A, lda, trans, i, p)) *
                               Fraction(_a(A, lda, trans, j, p))) for p in range(k)),
                          Fraction(0))
                bound = (k + 3) * U * (abs(Fraction(alpha)) * mag + abs(Fraction(beta) *
                                                                        Fraction(old)))
                assert abs(Fraction(got) - exact) <= bound, (uplo, trans, n, k, i, j)
            gap = C.reshape(n, ldc)[:, n:] if n else C[:0]
            gap0 = C0.reshape(n, ldc)[:, n:] if n else C0[:0]
            assert np.array_equal(np.isnan(gap), np.isnan(gap0))


def pin_handworked(syrk):
    # A (2 x 3, column-major, lda 2) = [[0, 2, 4], [1, 3, 5]]; A A^T = [[20, 26], [26, 35]].
    A = np.arange(6, dtype=np.float64)
    C = np.full(4, 7.0)
    assert syrk("L", "N", 2, 3, 1.0, A, 2, 0.0, C, 2) == 0
    assert C.tolist() == [20.0, 26.0, 7.0, 35.0]
    # the same A read as 'T' (A is k x n = 2 x 3): A^T A = [[1, 3, 5], [3, 13, 23], [5, 23, 41]]
    C = np.full(9, 1.0)
    assert syrk("U", "T", 3, 2, 2.0, A, 2, -1.0, C, 3) == 0
    want = np.array([[1, 3, 5], [3, 13, 23], [5, 23, 41]], dtype=np.float64) * 2 - 1
    got = C.reshape(3, 3).T
    for i, j in itertools.product(range(3), range(3)):
        assert got[i, j] == (want[i, j] if i <= j else 1.0)


def pin_integer_exact(syrk):
    rng = np.random.Generator(np.random.PCG64(2))
    for uplo, trans, (n, k) in itertools.product("LU", "NT", ((37, 29), (64, 130), (5, 300))):
        rows, cols = (n, k) if trans == "N" else (k, n)
        Ai = rng.integers(-4, 5, (rows, cols))
        A = np.asfortranarray(Ai.astype(np.float64)).reshape(-1, order="F")
        C0i = rng.integers(-4, 5, (n, n))
        C = np.asfortranarray(C0i.astype(np.float64)).reshape(-1, order="F")
        assert syrk(uplo, trans, n, k, 2.0, A, rows, 0.5, C, n) == 0
        M = Ai @ Ai.T if trans == "N" else Ai.T @ Ai
        want = np.where(_tri(uplo, n), 2 * M + 0.5 * C0i, C0i)
        assert np.array_equal(C.reshape(n, n).T, want)


def pin_reduces_to_gemm(syrk):
    rng = np.random.Generator(np.random.PCG64(3))
    for uplo, trans, (n, k, pad) in itertools.product("LU", "NT", ((33, 47, 3), (70, 9, 0))):
        rows, cols = (n, k) if trans == "N" else (k, n)
        lda, ldc = rows + pad, n + pad
        A = inputs.colmajor(rng, rows, cols, lda)
        C0 = inputs.colmajor(rng, n, n, ldc)
        C = C0.copy()
        assert syrk(uplo, trans, n, k, -1.25, A, lda, 0.75, C, ldc) == 0
        tb = "T" if trans == "N" else "N"
        G = oracle.gemm_result(trans, tb, n, n, k, -1.25, A, lda, A, lda, 0.75, C0, ldc)
        got = inputs.as_matrix(C, n, n, ldc)
        gem = inputs.as_matrix(G, n, n, ldc)
        mask = _tri(uplo, n)
        assert np.array_equal(got[mask].view(np.uint64), gem[mask].view(np.uint64))
        assert np.array_equal(got[~mask].view(np.uint64),
                              inputs.as_matrix(C0, n, n, ldc)[~mask].view(np.uint64))


def pin_blas_rules(syrk):
    A = np.ones(12)
    C = np.zeros(16)
    assert syrk("X", "N", 2, 2, 1.0, A, 2, 0.0, C, 2) == -1
    assert syrk("L", "Q", 2, 2, 1.0, A, 2, 0.0, C, 2) == -2
    assert syrk("L", "N", -1, 2, 1.0, A, 2, 0.0, C, 2) == -3
    assert syrk("L", "N", 2, -1, 1.0, A, 2, 0.0, C, 2) == -4
    assert syrk("L", "N", 3, 2, 1.0, A, 2, 0.0, C, 3) == -7
    assert syrk("L", "T", 2, 3, 1.0, A, 2, 0.0, C, 2) == -7
    assert syrk("U", "N", 3, 2, 1.0, A, 3, 0.0, C, 2) == -10
    # beta == 0: C not read (NaN does not propagate); alpha == 0: A not read
    An = np.full(12, np.nan)
    Cn = np.full(4, np.nan)
    assert syrk("L", "N", 2, 2, 1.0, np.arange(4.0), 2, 0.0, Cn, 2) == 0
    assert not np.isnan(Cn[[0, 1, 3]]).any() and np.isnan(Cn[2])
    Cb = np.full(4, 3.0)
    assert syrk("U", "T", 2, 3, 0.0, An, 3, 0.5, Cb, 2) == 0
    assert Cb.tolist() == [1.5, 3.0, 1.5, 1.5]
    Cq = np.full(4, 3.0)
    assert syrk("U", "N", 2, 0, 5.0, An, 2, 1.0, Cq, 2) == 0 and Cq.tolist() == [3.0] * 4


SYRK_PINS = [pin_bruteforce, pin_handworked, pin_integer_exact, pin_reduces_to_gemm,
             pin_blas_rules]


@pytest.mark.parametrize("pin", SYRK_PINS, ids=lambda f: f.__name__)
def test_syrk_oracle_pin(pin):
    pin(oracle.syrk)


MUTANTS = {
    "upper_for_lower": ("int64_t i0 = lower ? j : 0, i1 = lower ? n : j + 1;",
                        "int64_t i0 = lower ? 0 : j, i1 = lower ? j + 1 : n;"),
    "aj_reads_row_i": ("double aj = notrans ? A[j + p * lda] : A[p + j * lda];",
                       "double aj = notrans ? A[i + p * lda] : A[p + j * lda];"),
    "dropped_beta": ("if (beta != 0.0) v += beta * *c;", ""),
    "beta_zero_reads_C": ("if (beta != 0.0) v += beta * *c;", "v += beta * *c;"),
    "transpose_ignored": ("double ai = notrans ? A[i + p * lda] : A[p + i * lda];",
                          "double ai = A[i + p * lda];"),
    "last_k_dropped": ("for (int64_t p = 0; p < k; ++p) {", "for (int64_t p = 0; p + 1 < k; ++p) {"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_syrk_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    cpath = tmp_path / f"{name}.c"
    cpath.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-shared", "-fPIC",
                    str(cpath), "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    i64, dbl, ptr = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    lib.oracle_syrk.argtypes = [ctypes.c_char, ctypes.c_char, i64, i64, dbl, ptr, i64, dbl,
                                ptr, i64]
    lib.oracle_syrk.restype = ctypes.c_int

    def syrk(uplo, trans, n, k, alpha, A, lda, beta, C, ldc):
        def p(a):
            return a.ctypes.data_as(ctypes.c_void_p)
        return lib.oracle_syrk(uplo.encode(), trans.encode(), n, k, float(alpha), p(A), lda,
                               float(beta), p(C), ldc)
    for pin in SYRK_PINS:
        try:
            with np.errstate(all="ignore"):
                pin(syrk)
        except (AssertionError, ValueError, IndexError):
            return
    pytest.fail(f"mutant {name} passed every pin")
