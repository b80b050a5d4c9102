"""Checks that pin the CPU oracle to facts outside itself.

Each ``pin_*`` function takes a ``gemm`` callable with the oracle's signature
``gemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, nthreads) -> info`` and
raises ``AssertionError`` when the callable disagrees with:

* exact rational arithmetic (``fractions.Fraction``) on tiny inputs, within the rounding
  bound of a k-term sum plus the alpha/beta scaling (brute force on tiny inputs);
* hand-derived worked examples (``tests/golden/textbook_products.txt``);
* closed forms: identity, permutation and rank-1 operands;
* exact integer matrix products computed by numpy's int64 matmul (a library routine);
* numpy's float64 matmul (an independent library routine) within the error bound;
* the BLAS rules of dgemm (argument codes, quick returns, beta == 0 and alpha == 0 not
  reading their operand, rows m..ldc-1 of C untouched).

The same battery runs against deliberately broken copies of the oracle (see
``test_oracle_mutants.py``) to show that a plausible mistake fails at least one pin.
"""
from __future__ import annotations

from fractions import Fraction
import itertools
import os

import numpy as np

from paper_2302_08417_gb300 import inputs

U64 = 2.0 ** -53
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "textbook_products.txt")


def _run(gemm, p: inputs.Problem, C=None):
    C = np.array(p.C0 if C is None else C, dtype=np.float64, copy=True)
    info = gemm(p.transa, p.transb, p.m, p.n, p.k, p.alpha, p.A.astype(np.float64), p.lda,
                p.B.astype(np.float64), p.ldb, p.beta, C, p.ldc, 1)
    assert info == 0, f"info {info}"
    return C


def _opa(p):
    a = inputs.as_matrix(p.A.astype(np.float64), p.rows_a, p.cols_a, p.lda)
    return a if inputs.is_notrans(p.transa) else a.T


def _opb(p):
    b = inputs.as_matrix(p.B.astype(np.float64), p.rows_b, p.cols_b, p.ldb)
    return b if inputs.is_notrans(p.transb) else b.T


def _exact(p):
    """Exact rational alpha*op(A)op(B) + beta*C0 (the definition, in Fractions)."""
    opa, opb = _opa(p), _opb(p)
    c0 = inputs.as_matrix(p.C0.astype(np.float64), p.m, p.n, p.ldc)
    out = [[Fraction(0)] * p.n for _ in range(p.m)]
    absv = [[Fraction(0)] * p.n for _ in range(p.m)]
    al, be = Fraction(p.alpha), Fraction(p.beta)
    for i in range(p.m):
        for j in range(p.n):
            s = Fraction(0)
            sa = Fraction(0)
            for q in range(p.k):
                a, b = Fraction(float(opa[i, q])), Fraction(float(opb[q, j]))
                s += a * b
                sa += abs(a) * abs(b)
            v = al * s
            av = abs(al) * sa
            if p.beta != 0:
                cv = Fraction(float(c0[i, j]))
                v += be * cv
                av += abs(be) * abs(cv)
            out[i][j] = v
            absv[i][j] = av
    return out, absv


def pin_fraction_bruteforce(gemm, sizes=(0, 1, 2, 3, 5), trans="NTc"):
    """|oracle - exact| <= (k+3) u (|alpha||A||B| + |beta||C0|) on tiny shapes, all trans and
    leading-dimension combinations."""
    seed = 0
    for ta, tb in itertools.product(trans, trans):
        for m, n, k in itertools.product(sizes, sizes, sizes):
            for pad, (alpha, beta) in itertools.product(
                    (0, 3), ((1.0, 0.0), (-0.75, 0.5), (1.0, -1.25), (0.0, 0.5))):
                seed += 1
                p = inputs.problem(seed, ta, tb, m, n, k, alpha, beta, pad, pad, pad)
                C = _run(gemm, p)
                got = inputs.as_matrix(C, m, n, p.ldc)
                ex, absv = _exact(p)
                for i in range(m):
                    for j in range(n):
                        err = abs(Fraction(float(got[i, j])) - ex[i][j])
                        bound = Fraction((k + 3) * U64) * absv[i][j]
                        assert err <= bound, (ta, tb, m, n, k, alpha, beta, pad, i, j)
                # the gap rows of C keep their sentinel
                gap = C.reshape(max(n, 1), p.ldc)[:, m:] if n else C[:0]
                assert np.all(np.isnan(gap)), "C gap rows written"


def _parse_golden():
    cases = []
    with open(GOLDEN) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.lstrip().startswith("#")]
    i = 0
    while i < len(lines):
        head = lines[i].split()
        assert head[0] == "case", head
        name, ta, tb = head[1], head[2], head[3]
        m, n, k = int(head[4]), int(head[5]), int(head[6])
        alpha, beta = float(head[7]), float(head[8])
        i += 1
        blocks = {}
        shapes = {"A": (m, k) if ta == "N" else (k, m), "B": (k, n) if tb == "N" else (n, k),
                  "C0": (m, n), "C": (m, n)}
        for key in ("A", "B", "C0", "C"):
            assert lines[i] == key, (name, key, lines[i])
            i += 1
            r, c = shapes[key]
            rows = [[float(x) for x in lines[i + t].split()] for t in range(r)]
            i += r
            blocks[key] = np.array(rows, dtype=np.float64).reshape(r, c)
        cases.append((name, ta, tb, m, n, k, alpha, beta, blocks))
    return cases


def golden_cases():
    return _parse_golden()


def _flat(mat, ld):
    r, c = mat.shape
    buf = np.full((c, ld), np.nan)
    buf[:, :r] = mat.T
    return buf.reshape(-1).copy()


def pin_golden(gemm):
    """The hand-derived textbook products, bit-exact, with the operands stored at ld = rows
    and at ld = rows + 2 (NaN in the gap)."""
    for name, ta, tb, m, n, k, alpha, beta, bl in _parse_golden():
        for pad in (0, 2):
            ra, rb = bl["A"].shape[0], bl["B"].shape[0]
            lda, ldb, ldc = ra + pad, rb + pad, m + pad
            A, B, C = _flat(bl["A"], lda), _flat(bl["B"], ldb), _flat(bl["C0"], ldc)
            info = gemm(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, 1)
            assert info == 0
            got = inputs.as_matrix(C, m, n, ldc)
            assert np.array_equal(got, bl["C"]), (name, pad, got, bl["C"])


def pin_closed_forms(gemm):
    """op(A) = I gives alpha*op(B) + beta*C0 (two IEEE roundings, as numpy does them);
    op(A) = P (a permutation) permutes the rows of op(B); B = I gives alpha*op(A) + beta*C0;
    rank-1 integer operands A = u v^T, B = w z^T give (v.w) u z^T exactly."""
    rng = np.random.Generator(np.random.PCG64(7))
    for ta, tb in itertools.product("NT", "NT"):
        m, n = 7, 5
        k = m
        for alpha, beta in ((1.0, 0.0), (-0.75, 0.5), (2.0, 1.0)):
            p = inputs.problem(11, ta, tb, m, n, k, alpha, beta, 2, 3, 1)
            perm = rng.permutation(m)
            P = np.eye(m)[perm]              # (P X)[i] = X[perm[i]]
            stored = P if inputs.is_notrans(ta) else P.T
            p.A = _flat(stored, p.lda)
            C = _run(gemm, p)
            got = inputs.as_matrix(C, m, n, p.ldc)
            c0 = inputs.as_matrix(p.C0, m, n, p.ldc)
            want = alpha * _opb(p)[perm, :]
            if beta != 0.0:
                want = want + beta * c0
            assert np.array_equal(got, want), ("perm", ta, tb, alpha, beta)
            eye = np.eye(m)
            p.A = _flat(eye, p.lda)
            C = _run(gemm, p)
            want = alpha * _opb(p)
            if beta != 0.0:
                want = want + beta * c0
            assert np.array_equal(inputs.as_matrix(C, m, n, p.ldc), want), ("I", ta, tb)
        # B = I (k = n)
        m, n = 6, 4
        p = inputs.problem(12, ta, tb, m, n, n, -1.5, 0.25, 1, 2, 0)
        p.B = _flat(np.eye(n), p.ldb)
        C = _run(gemm, p)
        want = -1.5 * _opa(p) + 0.25 * inputs.as_matrix(p.C0, m, n, p.ldc)
        assert np.array_equal(inputs.as_matrix(C, m, n, p.ldc), want), ("B=I", ta, tb)
        # rank one
        m, n, k = 9, 6, 4
        u = rng.integers(-5, 6, m).astype(np.float64)
        v = rng.integers(-5, 6, k).astype(np.float64)
        w = rng.integers(-5, 6, k).astype(np.float64)
        z = rng.integers(-5, 6, n).astype(np.float64)
        opa, opb = np.outer(u, v), np.outer(w, z)
        p = inputs.problem(13, ta, tb, m, n, k, 1.0, 0.0, 1, 0, 2)
        p.A = _flat(opa if ta == "N" else opa.T, p.lda)
        p.B = _flat(opb if tb == "N" else opb.T, p.ldb)
        C = _run(gemm, p)
        want = float(v @ w) * np.outer(u, z)
        assert np.array_equal(inputs.as_matrix(C, m, n, p.ldc), want), ("rank1", ta, tb)


def pin_integer_exact(gemm):
    """Integer operands: the oracle equals numpy's exact int64 product bit for bit."""
    for seed, (ta, tb) in enumerate(itertools.product("NTc", "nTC")):
        for (m, n, k), (alpha, beta) in itertools.product(
                ((13, 11, 17), (1, 9, 33), (16, 1, 5), (4, 4, 64)),
                ((1.0, 0.0), (2.0, 3.0), (-1.0, -2.0), (1.0, 1.0))):
            p = inputs.problem(100 + seed, ta, tb, m, n, k, alpha, beta, 1, 7, 3,
                               dist="int", int_lim=8)
            C = _run(gemm, p)
            opa = _opa(p).astype(np.int64)
            opb = _opb(p).astype(np.int64)
            c0 = inputs.as_matrix(p.C0, m, n, p.ldc)
            want = int(alpha) * (opa @ opb)
            if beta != 0.0:
                want = want + int(beta) * np.nan_to_num(c0).astype(np.int64)
            assert np.array_equal(inputs.as_matrix(C, m, n, p.ldc), want.astype(np.float64)), \
                (ta, tb, m, n, k, alpha, beta)


def pin_numpy_matmul(gemm):
    """uniform[-1, 1] operands: within 2(k+2)u(|alpha||A||B| + |beta||C0|) of numpy's
    float64 matmul (an independently blocked library product)."""
    for seed, (ta, tb) in enumerate(itertools.product("NT", "NT")):
        for m, n, k in ((37, 29, 61), (64, 64, 64), (5, 70, 130)):
            for alpha, beta in ((1.0, 0.5), (-2.0, 0.0)):
                p = inputs.problem(200 + seed, ta, tb, m, n, k, alpha, beta, 7, 7, 7)
                C = _run(gemm, p)
                got = inputs.as_matrix(C, m, n, p.ldc)
                c0 = inputs.as_matrix(p.C0, m, n, p.ldc)
                ref = alpha * (_opa(p) @ _opb(p))
                absv = abs(alpha) * (np.abs(_opa(p)) @ np.abs(_opb(p)))
                if beta != 0.0:
                    ref = ref + beta * c0
                    absv = absv + abs(beta) * np.abs(c0)
                tol = 2 * (k + 2) * U64 * absv
                assert np.all(np.abs(got - ref) <= tol), (ta, tb, m, n, k)


def pin_blas_rules(gemm):
    """Argument codes, quick returns, and operands that must not be read."""
    A = np.ones(64)
    B = np.ones(64)
    C = np.ones(64)
    bad = [
        (("X", "N", 2, 2, 2, 1.0, A, 2, B, 2, 0.0, C, 2), -1),
        (("N", "Q", 2, 2, 2, 1.0, A, 2, B, 2, 0.0, C, 2), -2),
        (("N", "N", -1, 2, 2, 1.0, A, 2, B, 2, 0.0, C, 2), -3),
        (("N", "N", 2, -1, 2, 1.0, A, 2, B, 2, 0.0, C, 2), -4),
        (("N", "N", 2, 2, -1, 1.0, A, 2, B, 2, 0.0, C, 2), -5),
        (("N", "N", 3, 2, 2, 1.0, A, 2, B, 2, 0.0, C, 3), -8),
        (("T", "N", 2, 2, 3, 1.0, A, 2, B, 3, 0.0, C, 2), -8),
        (("N", "N", 2, 2, 3, 1.0, A, 2, B, 2, 0.0, C, 2), -10),
        (("N", "T", 2, 3, 2, 1.0, A, 2, B, 2, 0.0, C, 2), -10),
        (("N", "N", 3, 2, 2, 1.0, A, 3, B, 2, 0.0, C, 2), -13),
        (("N", "N", 0, 0, 0, 1.0, A, 0, B, 1, 0.0, C, 1), -8),
    ]
    for args, code in bad:
        assert gemm(*args, 1) == code, (args[:5], code)
    # beta == 0: a NaN in C must not propagate
    p = inputs.problem(300, "N", "N", 5, 4, 3, 1.0, 0.0, 1, 1, 1)
    C = np.full_like(p.C0, np.nan)
    C = _run(gemm, p, C)
    assert not np.any(np.isnan(inputs.as_matrix(C, 5, 4, p.ldc)))
    # alpha == 0: A and B are not read (NaN operands), C := beta*C0
    for k in (0, 3):
        p = inputs.problem(301, "T", "N", 5, 4, k, 0.0, 0.5, 0, 0, 1)
        p.A = np.full_like(p.A, np.nan)
        p.B = np.full_like(p.B, np.nan)
        C = _run(gemm, p)
        want = 0.5 * inputs.as_matrix(p.C0, 5, 4, p.ldc)
        assert np.array_equal(inputs.as_matrix(C, 5, 4, p.ldc), want)
    # k == 0 with nonzero alpha: C := beta*C0, A and B not read
    p = inputs.problem(302, "N", "N", 3, 3, 0, 1.0, -2.0, 0, 0, 0)
    p.A = np.full(4, np.nan)
    p.B = np.full(4, np.nan)
    C = _run(gemm, p)
    assert np.array_equal(inputs.as_matrix(C, 3, 3, p.ldc),
                          -2.0 * inputs.as_matrix(p.C0, 3, 3, p.ldc))
    # alpha == 0 and beta == 1: C untouched bit for bit (NaN payloads included)
    p = inputs.problem(303, "N", "N", 4, 4, 4, 0.0, 1.0)
    C0 = p.C0.copy()
    C0[3] = np.nan
    C = _run(gemm, p, C0)
    assert np.array_equal(C.view(np.uint64), C0.view(np.uint64))
    # m == 0 or n == 0: nothing written
    for m, n in ((0, 4), (4, 0)):
        p = inputs.problem(304, "N", "N", m, n, 3, 1.0, 0.0)
        C = np.full(32, 7.0)
        info = gemm("N", "N", m, n, 3, 1.0, np.ones(32), max(1, m), np.ones(32), 3, 0.0, C,
                    max(1, m), 1)
        assert info == 0 and np.all(C == 7.0)


ALL_PINS = [pin_golden, pin_closed_forms, pin_integer_exact, pin_numpy_matmul,
            pin_blas_rules, pin_fraction_bruteforce]
