"""SYRK on the fused kernel (gfip_dsyrk / gfip_ssyrk) through the C ABI, against the SYRK
oracle: the requested triangle within 2 max(k, 2) u (|alpha||A||A^T| + |beta||C0|), the
other triangle and the ld gap of C untouched bit for bit, small integers bit-exact, and the
pack policies (one packed copy of A serving both operand roles, or none) bit-identical."""
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

OTHER = 1.0e30   # sentinel in the triangle that must not be touched (finite in FP32)


@pytest.fixture(scope="module")
def runner():
    import __graft_entry__
    __graft_entry__.build()
    return gu.Runner()


def make(seed, uplo, trans, n, k, pad, dtype, dist="uniform"):
    rng = np.random.Generator(np.random.PCG64(seed))
    rows, cols = (n, k) if trans == "N" else (k, n)
    lda, ldc = max(1, rows + pad), max(1, n + pad)
    A = inputs.colmajor(rng, rows, cols, lda, dtype, dist)
    C0 = inputs.colmajor(rng, n, n, ldc, dtype, dist)
    if n:
        M = C0.reshape(n, ldc)          # M[j, i] = C[i, j]
        i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        other = (i < j) if uplo == "L" else (i > j)
        M[:, :n][other.T] = OTHER
    return A, lda, C0, ldc


def run(runner, uplo, trans, n, k, alpha, A, lda, beta, C0, ldc, policy=g.GFIP_PACK_AUTO,
        expect=0):
    esz = A.dtype.itemsize
    dA = torch.from_numpy(A).to(runner.dev)
    Cbuf = np.concatenate([C0, np.full(gu.GUARD, np.nan, dtype=C0.dtype)])
    dC = torch.from_numpy(Cbuf).to(runner.dev)
    runner.h.set_pack_policy(policy)
    runner.h.ensure_syrk_workspace(uplo, trans, n, k, esz)
    rc = g.gfip_syrk(esz, runner.h.h, uplo, trans, n, k, alpha, dA.data_ptr(), lda, beta,
                     dC.data_ptr(), ldc)
    runner.h.set_pack_policy(g.GFIP_PACK_AUTO)
    assert rc == expect, g.error_string(rc)
    torch.cuda.synchronize()
    out = dC.cpu().numpy()
    assert runner.h.status() == 0
    return out[: C0.size], out[C0.size:]


def check(uplo, trans, n, k, alpha, A, lda, beta, C0, ldc, got, guard):
    A64, C064 = A.astype(np.float64), C0.astype(np.float64)
    ref = oracle.syrk_result(uplo, trans, n, k, alpha, A64, lda, beta, C064, ldc)
    u = inputs.unit_roundoff(A.dtype)
    gm = inputs.as_matrix(got.astype(np.float64), n, n, ldc)
    rm = inputs.as_matrix(ref, n, n, ldc)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    tri = (i >= j) if uplo == "L" else (i <= j)
    # the other triangle and the gap rows keep their bytes
    c0m = inputs.as_matrix(C0, n, n, ldc)
    assert np.array_equal(inputs.as_matrix(got, n, n, ldc)[~tri].view(np.uint8),
                          c0m[~tri].view(np.uint8))
    if n and ldc > n:
        assert np.array_equal(got.reshape(n, ldc)[:, n:].view(np.uint8),
                              C0.reshape(n, ldc)[:, n:].view(np.uint8))
    assert np.all(np.isnan(guard))
    if not tri.any():
        return
    tb = "T" if trans == "N" else "N"
    if alpha == 0.0 or k == 0:
        bound = np.abs(beta * inputs.as_matrix(C064, n, n, ldc))
    else:
        bound = oracle.abs_bound(trans, tb, n, n, k, alpha, A64, lda, A64, lda, beta, C064,
                                 ldc, nthreads=4)
    tol = 2.0 * max(k, 2) * u * bound
    err = np.abs(gm - rm)
    bad = tri & ~(err <= tol)
    assert not bad.any(), (uplo, trans, n, k, np.argwhere(bad)[0])


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("uplo,trans", list(itertools.product("LU", "NT")))
def test_tiny_bruteforce(runner, dtype, uplo, trans):
    for n, k, pad, beta in itertools.product((0, 1, 2, 3, 5, 8, 17, 33), (0, 1, 3, 16, 17),
                                             (0, 7), (0.0, 0.5)):
        A, lda, C0, ldc = make(n * 100 + k, uplo, trans, n, k, pad, dtype)
        got, guard = run(runner, uplo, trans, n, k, -1.5, A, lda, beta, C0, ldc)
        check(uplo, trans, n, k, -1.5, A, lda, beta, C0, ldc, got, guard)


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("uplo,trans", list(itertools.product("LU", "NT")))
def test_ragged_and_policies_bitwise(runner, dtype, uplo, trans):
    for n, k in ((100, 70), (257, 300), (700, 129)):
        A, lda, C0, ldc = make(n + k, uplo, trans, n, k, 7, dtype)
        first = None
        for policy in (g.GFIP_PACK_AUTO, g.GFIP_PACK_NONE, g.GFIP_PACK_BOTH):
            got, guard = run(runner, uplo, trans, n, k, 0.75, A, lda, 0.5, C0, ldc, policy)
            if first is None:
                check(uplo, trans, n, k, 0.75, A, lda, 0.5, C0, ldc, got, guard)
                first = got
            else:
                assert np.array_equal(got.view(np.uint8), first.view(np.uint8)), policy


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_integer_bit_exact(runner, dtype):
    for uplo, trans, (n, k) in itertools.product("LU", "NT", ((130, 90), (300, 1000))):
        A, lda, C0, ldc = make(7 + n, uplo, trans, n, k, 3, dtype, dist="int")
        for policy in (g.GFIP_PACK_NONE, g.GFIP_PACK_BOTH):
            got, _ = run(runner, uplo, trans, n, k, 2.0, A, lda, 0.5, C0, ldc, policy)
            ref = oracle.syrk_result(uplo, trans, n, k, 2.0, A.astype(np.float64), lda, 0.5,
                                     C0.astype(np.float64), ldc)
            assert np.array_equal(inputs.as_matrix(got.astype(np.float64), n, n, ldc),
                                  inputs.as_matrix(ref, n, n, ldc))


def test_blas_rules(runner):
    n, k = 70, 40
    A, lda, C0, ldc = make(3, "L", "N", n, k, 2, np.float64)
    # beta == 0: C not read (NaN in the triangle does not propagate)
    Cn = C0.copy()
    Cn[np.isfinite(Cn) & (Cn != OTHER)] = np.nan
    got, guard = run(runner, "L", "N", n, k, 1.0, A, lda, 0.0, Cn, ldc)
    tri = np.tril(np.ones((n, n), bool))
    assert not np.isnan(inputs.as_matrix(got, n, n, ldc)[tri]).any()
    # alpha == 0: A not read, C := beta C on the triangle only
    An = np.full_like(A, np.nan)
    got, guard = run(runner, "L", "N", n, k, 0.0, An, lda, 0.5, C0, ldc)
    check("L", "N", n, k, 0.0, A, lda, 0.5, C0, ldc, got, guard)
    # argument codes
    for args, code in (((b"X", b"N", 4, 4), -1), ((b"L", b"Q", 4, 4), -2),
                       ((b"L", b"N", -1, 4), -3), ((b"L", b"N", 4, -1), -4)):
        rc = g.load().gfip_dsyrk(runner.h.h, args[0], args[1], args[2], args[3], 1.0, None,
                                 max(1, args[2]), 0.0, None, max(1, args[2]))
        assert rc == code
    assert g.load().gfip_dsyrk(runner.h.h, b"L", b"N", 8, 4, 1.0, None, 7, 0.0, None, 8) == -7
    assert g.load().gfip_dsyrk(runner.h.h, b"U", b"T", 8, 4, 1.0, None, 4, 0.0, None, 7) == -10


@pytest.mark.parametrize("dtype,uplo,trans,n,k", [
    (np.float64, "L", "N", 4096, 2048),
    (np.float32, "U", "T", 8192, 1024),
])
def test_large_sampled(runner, dtype, uplo, trans, n, k):
    """Full-size shapes on sampled triangle entries (4096 random plus 4 whole columns)."""
    A, lda, C0, ldc = make(n + k, uplo, trans, n, k, 7, dtype)
    got, guard = run(runner, uplo, trans, n, k, 1.0, A, lda, 0.5, C0, ldc)
    assert np.all(np.isnan(guard))
    rng = np.random.Generator(np.random.PCG64(9))
    ii, jj = inputs.sample_indices(rng, n, n, 4096, full_cols=4)
    keep = (ii >= jj) if uplo == "L" else (ii <= jj)
    ii, jj = ii[keep], jj[keep]
    tb = "T" if trans == "N" else "N"
    A64, C064 = A.astype(np.float64), C0.astype(np.float64)
    args = (trans, tb, n, n, k, 1.0, A64, lda, A64, lda, 0.5, C064, ldc, ii, jj)
    want = oracle.entries(*args, nthreads=8)
    bound = oracle.entries(*args, absval=True, nthreads=8)
    gv = inputs.as_matrix(got, n, n, ldc)[ii, jj].astype(np.float64)
    assert np.all(np.abs(gv - want) <= 2 * k * inputs.unit_roundoff(A.dtype) * bound)
    # the other triangle untouched on the sampled mirror positions
    c0m = inputs.as_matrix(C0, n, n, ldc)
    off = jj != ii
    assert np.array_equal(inputs.as_matrix(got, n, n, ldc)[jj[off], ii[off]].view(np.uint8),
                          c0m[jj[off], ii[off]].view(np.uint8))
