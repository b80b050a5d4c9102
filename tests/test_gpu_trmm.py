"""TRMM on the fused kernel (gfip_dtrmm / gfip_strmm) through the C ABI, against the TRMM
oracle, for all 16 side / uplo / trans / diag combinations.  A carries NaN in every entry
TRMM must not read (the other triangle, and the diagonal when it is unit), so a mask that
lets one through shows up as NaN.  Bound: 2 max(k, 2) u |alpha| (|op(A)||B|) with op(A)
written out densely (zeros outside the triangle, ones on a unit diagonal), k the order of A;
small integers bit-exact; the pack policies (masked panels packed by the first tile line, or
none) bit-identical; the rows m..ldb-1 of B untouched."""
import itertools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2302_08417_gb300 import gemmfip as g  # noqa: E402
from paper_2302_08417_gb300 import inputs  # noqa: E402
from tests import gpu_util as gu  # noqa: E402

COMBOS = list(itertools.product("LR", "LU", "NT", "NU"))


@pytest.fixture(scope="module")
def runner():
    import __graft_entry__
    __graft_entry__.build()
    return gu.Runner()


def poisoned(rng, na, lda, uplo, diag, dtype, dist="uniform"):
    A = inputs.colmajor(rng, na, na, lda, dtype, dist)
    if na:
        M = A[: lda * na].reshape(na, lda)          # M[c, r] = A[r, c]
        r, c = np.meshgrid(np.arange(na), np.arange(na), indexing="ij")
        bad = (r < c) if uplo == "L" else (r > c)
        if diag == "U":
            bad |= r == c
        M[:, :na][bad.T] = np.nan
    return A


def dense_op(A, lda, na, uplo, transa, diag):
    S = inputs.as_matrix(A, na, na, lda).astype(np.float64)
    i, j = np.meshgrid(np.arange(na), np.arange(na), indexing="ij")
    keep = (i >= j) if uplo == "L" else (i <= j)
    if diag == "U":
        keep &= i != j
    D = np.where(keep, S, 0.0)
    if diag == "U":
        D[np.arange(na), np.arange(na)] = 1.0
    return D.T.copy() if transa != "N" else D


def run(runner, side, uplo, ta, diag, m, n, alpha, A, lda, B0, ldb, policy=g.GFIP_PACK_AUTO):
    esz = A.dtype.itemsize
    dA = torch.from_numpy(A).to(runner.dev)
    Bbuf = np.concatenate([B0, np.full(gu.GUARD, np.nan, dtype=B0.dtype)])
    dB = torch.from_numpy(Bbuf).to(runner.dev)
    runner.h.set_pack_policy(policy)
    runner.h.ensure_trmm_workspace(side, uplo, ta, diag, m, n, esz)
    rc = g.gfip_trmm(esz, runner.h.h, side, uplo, ta, diag, m, n, alpha, dA.data_ptr(), lda,
                     dB.data_ptr(), ldb)
    runner.h.set_pack_policy(g.GFIP_PACK_AUTO)
    assert rc == 0, g.error_string(rc)
    torch.cuda.synchronize()
    out = dB.cpu().numpy()
    assert runner.h.status() == 0
    return out[: B0.size], out[B0.size:]


def check(side, uplo, ta, diag, m, n, alpha, A, lda, B0, ldb, got, guard):
    na = m if side == "L" else n
    A64, B64 = A.astype(np.float64), B0.astype(np.float64)
    ref = oracle.trmm_result(side, uplo, ta, diag, m, n, alpha, A64, lda, B64, ldb)
    if m and ldb > m:
        assert np.array_equal(got.reshape(n, ldb)[:, m:].view(np.uint8),
                              B0.reshape(n, ldb)[:, m:].view(np.uint8))
    assert np.all(np.isnan(guard))
    if m == 0 or n == 0:
        return
    D = np.asfortranarray(dense_op(A64, lda, na, uplo, ta, diag)).reshape(-1, order="F")
    Z = np.zeros(m * n)
    if side == "L":
        bound = oracle.abs_bound("N", "N", m, n, m, alpha, D, na, B64, ldb, 0.0, Z, m)
    else:
        bound = oracle.abs_bound("N", "N", m, n, n, alpha, B64, ldb, D, na, 0.0, Z, m)
    u = inputs.unit_roundoff(A.dtype)
    gm = inputs.as_matrix(got.astype(np.float64), m, n, ldb)
    rm = inputs.as_matrix(ref, m, n, ldb)
    err = np.abs(gm - rm)
    bad = ~(err <= 2.0 * max(na, 2) * u * bound)
    assert not bad.any(), (side, uplo, ta, diag, m, n, np.argwhere(bad)[0])


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("side,uplo,ta,diag", COMBOS)
def test_bruteforce_small(runner, dtype, side, uplo, ta, diag):
    rng = np.random.Generator(np.random.PCG64(11))
    for (m, n), pad, alpha in itertools.product(((0, 3), (1, 1), (5, 3), (17, 33), (33, 17)),
                                                (0, 7), (1.0, -0.75)):
        na = m if side == "L" else n
        lda, ldb = max(1, na + pad), max(1, m + pad)
        A = poisoned(rng, na, lda, uplo, diag, dtype)
        B0 = inputs.colmajor(rng, m, n, ldb, dtype)
        got, guard = run(runner, side, uplo, ta, diag, m, n, alpha, A, lda, B0, ldb)
        check(side, uplo, ta, diag, m, n, alpha, A, lda, B0, ldb, got, guard)


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("side,uplo,ta,diag", COMBOS)
def test_ragged_and_policies_bitwise(runner, dtype, side, uplo, ta, diag):
    rng = np.random.Generator(np.random.PCG64(12))
    for m, n in ((300, 200), (130, 700)):
        na = m if side == "L" else n
        A = poisoned(rng, na, na + 3, uplo, diag, dtype)
        B0 = inputs.colmajor(rng, m, n, m + 5, dtype)
        first = None
        for policy in (g.GFIP_PACK_AUTO, g.GFIP_PACK_NONE, g.GFIP_PACK_BOTH):
            got, guard = run(runner, side, uplo, ta, diag, m, n, 1.25, A, na + 3, B0, m + 5,
                             policy)
            if first is None:
                check(side, uplo, ta, diag, m, n, 1.25, A, na + 3, B0, m + 5, got, guard)
                first = got
            else:
                assert np.array_equal(got.view(np.uint8), first.view(np.uint8)), policy


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_integer_bit_exact(runner, dtype):
    rng = np.random.Generator(np.random.PCG64(13))
    for side, uplo, ta, diag in COMBOS:
        m, n = 150, 90
        na = m if side == "L" else n
        A = poisoned(rng, na, na + 1, uplo, diag, dtype, dist="int")
        B0 = inputs.colmajor(rng, m, n, m + 2, dtype, dist="int")
        got, _ = run(runner, side, uplo, ta, diag, m, n, 2.0, A, na + 1, B0, m + 2,
                     g.GFIP_PACK_BOTH)
        ref = oracle.trmm_result(side, uplo, ta, diag, m, n, 2.0, A.astype(np.float64), na + 1,
                                 B0.astype(np.float64), m + 2)
        assert np.array_equal(inputs.as_matrix(got.astype(np.float64), m, n, m + 2),
                              inputs.as_matrix(ref, m, n, m + 2)), (side, uplo, ta, diag)


def test_alpha_zero_and_codes(runner):
    m, n = 40, 30
    A = np.full(m * m, np.nan)
    B0 = np.full(m * n, np.nan)
    got, _ = run(runner, "L", "U", "N", "N", m, n, 0.0, A, m, B0, m)
    assert np.all(got == 0.0)
    lib = g.load()
    for args, code in (((b"X", b"L", b"N", b"N", 2, 2, 2, 2), -1),
                       ((b"L", b"X", b"N", b"N", 2, 2, 2, 2), -2),
                       ((b"L", b"L", b"X", b"N", 2, 2, 2, 2), -3),
                       ((b"L", b"L", b"N", b"X", 2, 2, 2, 2), -4),
                       ((b"L", b"L", b"N", b"N", -1, 2, 2, 2), -5),
                       ((b"L", b"L", b"N", b"N", 2, -1, 2, 2), -6),
                       ((b"L", b"L", b"N", b"N", 3, 2, 2, 3), -9),
                       ((b"R", b"U", b"T", b"U", 3, 2, 2, 2), -11)):
        s_, u_, t_, d_, m_, n_, lda_, ldb_ = args
        assert lib.gfip_dtrmm(runner.h.h, s_, u_, t_, d_, m_, n_, 1.0, None, lda_, None,
                              ldb_) == code


@pytest.mark.parametrize("dtype,side,uplo,ta,diag,m,n", [
    (np.float64, "L", "L", "N", "N", 4096, 2048),
    (np.float32, "R", "U", "T", "U", 2048, 4096),
])
def test_large_sampled(runner, dtype, side, uplo, ta, diag, m, n):
    """Full-size shapes on sampled entries (4096 random plus 4 whole rows and columns)."""
    rng = np.random.Generator(np.random.PCG64(14))
    na = m if side == "L" else n
    A = poisoned(rng, na, na + 7, uplo, diag, dtype)
    B0 = inputs.colmajor(rng, m, n, m + 7, dtype)
    got, guard = run(runner, side, uplo, ta, diag, m, n, 1.0, A, na + 7, B0, m + 7)
    assert np.all(np.isnan(guard))
    D = np.asfortranarray(dense_op(A.astype(np.float64), na + 7, na, uplo, ta, diag))
    D = D.reshape(-1, order="F")
    B64 = B0.astype(np.float64)
    ii, jj = inputs.sample_indices(rng, m, n, 4096, full_rows=4, full_cols=4)
    if side == "L":
        args = ("N", "N", m, n, m, 1.0, D, na, B64, m + 7, 0.0, None, m, ii, jj)
    else:
        args = ("N", "N", m, n, n, 1.0, B64, m + 7, D, na, 0.0, None, m, ii, jj)
    want = oracle.entries(*args, nthreads=8)
    bound = oracle.entries(*args, absval=True, nthreads=8)
    gv = inputs.as_matrix(got, m, n, m + 7)[ii, jj].astype(np.float64)
    assert np.all(np.abs(gv - want) <= 2 * na * inputs.unit_roundoff(A.dtype) * bound)
