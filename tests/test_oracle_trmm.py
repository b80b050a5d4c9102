"""Pins of the TRMM oracle (oracle/trmm_oracle.c) against what the definition and the
mathematics fix, and planted mistakes that must fail them.  CPU only.

* exact rational brute force (fractions.Fraction) on tiny shapes, all 16 side / uplo / trans
  / diag combinations, with NaN in every entry of A that must not be read;
* a hand-worked product, bit-exact;
* integer operands: exact against numpy's int64 product with the dense triangular matrix;
* the reduction to the (separately pinned) GEMM oracle: with op(A) written out as a dense
  matrix (zeros outside the triangle, ones on a unit diagonal) the GEMM gives the same values;
* reference-BLAS rules: argument codes, alpha == 0 (B := 0, neither A nor B read)."""
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
                   "trmm_oracle.c")
COMBOS = list(itertools.product("LR", "LU", "NT", "NU"))


def dense_op(A, lda, na, uplo, transa, diag):
    """op(A) as a dense na x na float64 matrix: zeros outside its triangle, ones on a unit
    diagonal (the stored A is read only where TRMM reads it)."""
    S = inputs.as_matrix(A, na, na, lda).astype(np.float64)
    i, j = np.meshgrid(np.arange(na), np.arange(na), indexing="ij")
    keep = (i >= j) if uplo == "L" else (i <= j)
    if diag == "U":
        keep &= i != j
    D = np.where(keep, S, 0.0)
    if diag == "U":
        D[np.arange(na), np.arange(na)] = 1.0
    return D.T.copy() if transa != "N" else D


def poison(A, lda, na, uplo, diag):
    """A copy of A with NaN everywhere TRMM must not read."""
    P = A.copy()
    M = P[: lda * na].reshape(na, lda) if na else P[:0]
    for c, r in itertools.product(range(na), range(na)):
        inside = (r >= c) if uplo == "L" else (r <= c)
        if not inside or (diag == "U" and r == c):
            M[c, r] = np.nan
    return P


def pin_bruteforce(trmm):
    rng = np.random.Generator(np.random.PCG64(4))
    for (side, uplo, ta, diag), (m, n), pad in itertools.product(
            COMBOS, ((0, 2), (1, 1), (2, 3), (3, 2), (4, 4)), (0, 2)):
        na = m if side == "L" else n
        lda, ldb = max(1, na + pad), max(1, m + pad)
        A = poison(inputs.colmajor(rng, na, na, lda), lda, na, uplo, diag)
        B0 = inputs.colmajor(rng, m, n, ldb)
        for alpha in (1.0, -0.75):
            B = B0.copy()
            assert trmm(side, uplo, ta, diag, m, n, alpha, A, lda, B, ldb) == 0
            D = dense_op(A, lda, na, uplo, ta, diag) if na else np.zeros((0, 0))
            Bm = inputs.as_matrix(B0, m, n, ldb)
            for i, j in itertools.product(range(m), range(n)):
                if side == "L":
                    terms = [Fraction(D[i, p]) * Fraction(Bm[p, j]) for p in range(m)
                             if D[i, p] != 0 or (diag == "U" and p == i)]
                else:
                    terms = [Fraction(Bm[i, p]) * Fraction(D[p, j]) for p in range(n)
                             if D[p, j] != 0 or (diag == "U" and p == j)]
                exact = Fraction(alpha) * sum(terms, Fraction(0))
                mag = abs(Fraction(alpha)) * sum((abs(t) for t in terms), Fraction(0))
                got = B[i + j * ldb]
                assert np.isfinite(got)
                assert abs(Fraction(got) - exact) <= (na + 2) * U * mag, (side, uplo, ta, diag)
            if m and ldb > m:
                assert np.isnan(B.reshape(n, ldb)[:, m:]).all()


def pin_handworked(trmm):
    # A = [[2, 9], [3, 5]] (column-major [2, 3, 9, 5]); lower non-unit op(A) = [[2, 0], [3, 5]]
    A = np.array([2.0, 3.0, 9.0, 5.0])
    B = np.array([1.0, 2.0, 4.0, -1.0])          # B = [[1, 4], [2, -1]]
    assert trmm("L", "L", "N", "N", 2, 2, 1.0, A, 2, B, 2) == 0
    assert B.tolist() == [2.0, 13.0, 8.0, 7.0]   # [[2, 8], [13, 7]]
    # upper unit, transposed, right side: op(A) = ([[1, 9], [0, 1]])^T = [[1, 0], [9, 1]]
    B = np.array([1.0, 2.0, 4.0, -1.0])
    assert trmm("R", "U", "T", "U", 2, 2, 2.0, A, 2, B, 2) == 0
    # B op(A) = [[1 + 36, 4], [2 - 9, -1]] = [[37, 4], [-7, -1]], times 2
    assert B.tolist() == [74.0, -14.0, 8.0, -2.0]


def pin_integer_exact(trmm):
    rng = np.random.Generator(np.random.PCG64(5))
    for (side, uplo, ta, diag), (m, n) in itertools.product(COMBOS, ((37, 23), (64, 70))):
        na = m if side == "L" else n
        Ai = rng.integers(-4, 5, (na, na))
        Bi = rng.integers(-4, 5, (m, n))
        A = np.asfortranarray(Ai.astype(np.float64)).reshape(-1, order="F")
        B = np.asfortranarray(Bi.astype(np.float64)).reshape(-1, order="F")
        assert trmm(side, uplo, ta, diag, m, n, 2.0, A, na, B, m) == 0
        D = dense_op(A, na, na, uplo, ta, diag).astype(np.int64)
        want = 2 * (D @ Bi if side == "L" else Bi @ D)
        assert np.array_equal(B.reshape(n, m).T, want)


def pin_reduces_to_gemm(trmm):
    rng = np.random.Generator(np.random.PCG64(6))
    for (side, uplo, ta, diag), (m, n, pad) in itertools.product(COMBOS, ((33, 20, 3),)):
        na = m if side == "L" else n
        lda, ldb = na + pad, m + pad
        A = inputs.colmajor(rng, na, na, lda)
        B0 = inputs.colmajor(rng, m, n, ldb)
        B = B0.copy()
        assert trmm(side, uplo, ta, diag, m, n, -1.5, A, lda, B, ldb) == 0
        D = np.asfortranarray(dense_op(A, lda, na, uplo, ta, diag)).reshape(-1, order="F")
        Z = np.zeros(m * n)
        if side == "L":
            G = oracle.gemm_result("N", "N", m, n, m, -1.5, D, na, B0, ldb, 0.0, Z, m)
        else:
            G = oracle.gemm_result("N", "N", m, n, n, -1.5, B0, ldb, D, na, 0.0, Z, m)
        assert np.array_equal(inputs.as_matrix(B, m, n, ldb), inputs.as_matrix(G, m, n, m))


def pin_blas_rules(trmm):
    A = np.ones(16)
    B = np.ones(16)
    assert trmm("X", "L", "N", "N", 2, 2, 1.0, A, 2, B, 2) == -1
    assert trmm("L", "X", "N", "N", 2, 2, 1.0, A, 2, B, 2) == -2
    assert trmm("L", "L", "X", "N", 2, 2, 1.0, A, 2, B, 2) == -3
    assert trmm("L", "L", "N", "X", 2, 2, 1.0, A, 2, B, 2) == -4
    assert trmm("L", "L", "N", "N", -1, 2, 1.0, A, 2, B, 2) == -5
    assert trmm("L", "L", "N", "N", 2, -1, 1.0, A, 2, B, 2) == -6
    assert trmm("L", "L", "N", "N", 3, 2, 1.0, A, 2, B, 3) == -9
    assert trmm("R", "L", "N", "N", 2, 3, 1.0, A, 2, B, 2) == -9
    assert trmm("R", "U", "T", "U", 3, 2, 1.0, A, 2, B, 2) == -11
    # alpha == 0: B := 0 without reading A or B
    Bn = np.full(4, np.nan)
    assert trmm("L", "U", "N", "N", 2, 2, 0.0, np.full(4, np.nan), 2, Bn, 2) == 0
    assert Bn.tolist() == [0.0] * 4


TRMM_PINS = [pin_bruteforce, pin_handworked, pin_integer_exact, pin_reduces_to_gemm,
             pin_blas_rules]


@pytest.mark.parametrize("pin", TRMM_PINS, ids=lambda f: f.__name__)
def test_trmm_oracle_pin(pin):
    pin(oracle.trmm)


MUTANTS = {
    "unit_diag_read": ("if (r == c && unit) return 1.0;", ""),
    "triangle_swapped": ("*nz = lower_op ? (r >= c) : (r <= c);",
                         "*nz = lower_op ? (r <= c) : (r >= c);"),
    "transpose_ignored": ("return trans ? A[c + r * lda] : A[r + c * lda];",
                          "return A[r + c * lda];"),
    "alpha_dropped": ("B[i + j * ldb] = alpha * s;\n            }\n        }\n        free(col);",
                      "B[i + j * ldb] = s;\n            }\n        }\n        free(col);"),
    "in_place_left": ("if (nz) s += a * col[p];", "if (nz) s += a * B[p + j * ldb];"),
    "strict_triangle": ("*nz = lower_op ? (r >= c) : (r <= c);",
                        "*nz = lower_op ? (r > c) : (r < c);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_trmm_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    cpath = tmp_path / f"{name}.c"
    cpath.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-shared", "-fPIC",
                    str(cpath), "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    i64, dbl, ptr, ch = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_char
    lib.oracle_trmm.argtypes = [ch, ch, ch, ch, i64, i64, dbl, ptr, i64, ptr, i64]
    lib.oracle_trmm.restype = ctypes.c_int

    def trmm(side, uplo, ta, diag, m, n, alpha, A, lda, B, ldb):
        def p(a):
            return a.ctypes.data_as(ctypes.c_void_p)
        return lib.oracle_trmm(side.encode(), uplo.encode(), ta.encode(), diag.encode(), m, n,
                               float(alpha), p(A), lda, p(B), ldb)
    for pin in TRMM_PINS:
        try:
            with np.errstate(all="ignore"):
                pin(trmm)
        except (AssertionError, ValueError, IndexError):
            return
    pytest.fail(f"mutant {name} passed every pin")
