"""Pins of the TRSM oracle (oracle/trsm_oracle.c) against what the mathematics fixes, and
planted mistakes that must fail them.  CPU only.

* the componentwise residual bound of substitution, checked in exact rational arithmetic on
  tiny shapes, all 16 side / uplo / trans / diag combinations, with NaN in every entry of A
  that must not be read: |op(A) X - alpha B| <= (k + 2) u (|op(A)| |X| + |alpha B|) (the
  computed solution of a triangular system solves a nearby system, |dT| <= k u |T|);
* integer systems with a unit diagonal have integer solutions: exact against an integer
  substitution in Python;
* TRSM undoes TRMM (the separately pinned TRMM oracle): bit-exact on integer unit systems;
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
from tests.test_oracle_trmm import dense_op, poison

U = 2.0 ** -53
SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "trsm_oracle.c")
COMBOS = list(itertools.product("LR", "LU", "NT", "NU"))


def dominant(rng, na, lda):
    """U[-1, 1] off the diagonal, diagonal of magnitude 1 + na (well conditioned)."""
    A = inputs.colmajor(rng, na, na, lda)
    for i in range(na):
        A[i + i * lda] = (1.0 + na) * (1 if rng.random() < 0.5 else -1)
    return A


def pin_residual(trsm):
    rng = np.random.Generator(np.random.PCG64(7))
    for (side, uplo, ta, diag), (m, n), pad in itertools.product(
            COMBOS, ((0, 2), (1, 1), (2, 3), (3, 2), (4, 4)), (0, 2)):
        na = m if side == "L" else n
        lda, ldb = max(1, na + pad), max(1, m + pad)
        A = poison(dominant(rng, na, lda), lda, na, uplo, diag)
        B0 = inputs.colmajor(rng, m, n, ldb)
        for alpha in (1.0, -0.75):
            X = B0.copy()
            assert trsm(side, uplo, ta, diag, m, n, alpha, A, lda, X, ldb) == 0
            if m == 0 or n == 0:
                continue
            D = dense_op(A, lda, na, uplo, ta, diag)
            Xm = inputs.as_matrix(X, m, n, ldb)
            Bm = inputs.as_matrix(B0, m, n, ldb)
            assert np.isfinite(Xm).all()
            for i, j in itertools.product(range(m), range(n)):
                if side == "L":
                    pairs = [(D[i, p], Xm[p, j]) for p in range(m)]
                else:
                    pairs = [(Xm[i, p], D[p, j]) for p in range(n)]
                r = sum((Fraction(a) * Fraction(b) for a, b in pairs), Fraction(0))
                r -= Fraction(alpha) * Fraction(Bm[i, j])
                mag = sum((abs(Fraction(a) * Fraction(b)) for a, b in pairs), Fraction(0))
                mag += abs(Fraction(alpha) * Fraction(Bm[i, j]))
                assert abs(r) <= (na + 2) * U * mag, (side, uplo, ta, diag, m, n, i, j)
            if ldb > m:
                assert np.isnan(X.reshape(n, ldb)[:, m:]).all()


def _int_solve(D, Bi, side):
    """Exact integer substitution for a unit triangular D (Python ints)."""
    na = D.shape[0]
    T = D if side == "L" else D.T
    lower = np.all(np.triu(T, 1) == 0)
    R = Bi if side == "L" else Bi.T
    X = [[0] * R.shape[1] for _ in range(na)]
    order = range(na) if lower else range(na - 1, -1, -1)
    for v in range(R.shape[1]):
        for i in order:
            s = int(R[i, v])
            for c in range(na):
                if c != i and T[i, c] != 0:
                    s -= int(T[i, c]) * X[c][v]
            X[i][v] = s
    X = np.array(X, dtype=object)
    return X if side == "L" else X.T


def pin_integer_unit(trsm):
    rng = np.random.Generator(np.random.PCG64(8))
    for (side, uplo, ta), (m, n) in itertools.product(
            itertools.product("LR", "LU", "NT"), ((9, 5), (6, 11))):
        na = m if side == "L" else n
        Ai = rng.integers(-1, 2, (na, na))
        Bi = rng.integers(-3, 4, (m, n))
        A = np.asfortranarray(Ai.astype(np.float64)).reshape(-1, order="F")
        X = np.asfortranarray(Bi.astype(np.float64)).reshape(-1, order="F")
        assert trsm(side, uplo, ta, "U", m, n, 1.0, A, na, X, m) == 0
        D = dense_op(A, na, na, uplo, ta, "U").astype(np.int64)
        want = _int_solve(D, Bi, side)
        assert np.array_equal(X.reshape(n, m).T, want.astype(np.float64)), (side, uplo, ta)


def pin_undoes_trmm(trsm):
    rng = np.random.Generator(np.random.PCG64(9))
    for (side, uplo, ta), (m, n) in itertools.product(
            itertools.product("LR", "LU", "NT"), ((13, 7), (8, 16))):
        na = m if side == "L" else n
        A = np.asfortranarray(rng.integers(-1, 2, (na, na)).astype(np.float64))
        A = A.reshape(-1, order="F")
        B0 = np.asfortranarray(rng.integers(-4, 5, (m, n)).astype(np.float64))
        B0 = B0.reshape(-1, order="F")
        Y = oracle.trmm_result(side, uplo, ta, "U", m, n, 1.0, A, na, B0, m)
        X = Y.copy()
        assert trsm(side, uplo, ta, "U", m, n, 1.0, A, na, X, m) == 0
        assert np.array_equal(X, B0), (side, uplo, ta)


def pin_blas_rules(trsm):
    A = np.ones(16)
    B = np.ones(16)
    assert trsm("X", "L", "N", "N", 2, 2, 1.0, A, 2, B, 2) == -1
    assert trsm("L", "X", "N", "N", 2, 2, 1.0, A, 2, B, 2) == -2
    assert trsm("L", "L", "X", "N", 2, 2, 1.0, A, 2, B, 2) == -3
    assert trsm("L", "L", "N", "X", 2, 2, 1.0, A, 2, B, 2) == -4
    assert trsm("L", "L", "N", "N", -1, 2, 1.0, A, 2, B, 2) == -5
    assert trsm("L", "L", "N", "N", 2, -1, 1.0, A, 2, B, 2) == -6
    assert trsm("L", "L", "N", "N", 3, 2, 1.0, A, 2, B, 3) == -9
    assert trsm("R", "U", "T", "U", 3, 2, 1.0, A, 2, B, 2) == -11
    Bn = np.full(4, np.nan)
    assert trsm("R", "L", "T", "N", 2, 2, 0.0, np.full(4, np.nan), 2, Bn, 2) == 0
    assert Bn.tolist() == [0.0] * 4


TRSM_PINS = [pin_residual, pin_integer_unit, pin_undoes_trmm, pin_blas_rules]


@pytest.mark.parametrize("pin", TRSM_PINS, ids=lambda f: f.__name__)
def test_trsm_oracle_pin(pin):
    pin(oracle.trsm)


MUTANTS = {
    "order_reversed": ("int64_t i = lower_t ? q : na - 1 - q;",
                       "int64_t i = lower_t ? na - 1 - q : q;"),
    "no_division": ("s = s / t;", "s = s;"),
    "alpha_dropped": ("(alpha == 0.0) ? 0.0 : alpha * B[i + j * ldb];",
                      "(alpha == 0.0) ? 0.0 : B[i + j * ldb];"),
    "side_transpose_lost": ("double t = left ? opa_el(A, lda, tt, i, c) : opa_el(A, lda, tt, c, i);",
                            "double t = opa_el(A, lda, tt, i, c);"),
    "unit_divides": ("if (!unit) {", "if (1) {"),
    "sum_sign": ("s -= t * base[c * step];", "s += t * base[c * step];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_trsm_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    cpath = tmp_path / f"{name}.c"
    cpath.write_text(src.replace(old, new))
    # the mutant is pinned on its own; TRMM (for the round trip) comes from the real oracle
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-shared", "-fPIC",
                    str(cpath), "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    i64, dbl, ptr, ch = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_char
    lib.oracle_trsm.argtypes = [ch, ch, ch, ch, i64, i64, dbl, ptr, i64, ptr, i64]
    lib.oracle_trsm.restype = ctypes.c_int

    def trsm(side, uplo, ta, diag, m, n, alpha, A, lda, B, ldb):
        def p(a):
            return a.ctypes.data_as(ctypes.c_void_p)
        return lib.oracle_trsm(side.encode(), uplo.encode(), ta.encode(), diag.encode(), m, n,
                               float(alpha), p(A), lda, p(B), ldb)
    for pin in TRSM_PINS:
        try:
            with np.errstate(all="ignore"):
                pin(trsm)
        except (AssertionError, ValueError, IndexError):
            return
    pytest.fail(f"mutant {name} passed every pin")
