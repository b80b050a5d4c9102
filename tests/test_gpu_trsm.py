"""TRSM on the fused kernel (gfip_dtrsm / gfip_strsm) through the C ABI, all 16 side / uplo /
trans / diag combinations, against what a triangular solve must satisfy: the componentwise
residual bound |op(A) X - alpha B| <= c u (|op(A)| |X| + |alpha B|) with c = 2 (k + 64) + 4
(substitution and the blocked GEMM updates each solve a nearby system), the oracle's
solution on well-conditioned systems, exact integer solutions of unit systems, and NaN in
every entry of A that must not be read."""
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
from tests.test_gpu_trmm import dense_op  # noqa: E402

COMBOS = list(itertools.product("LR", "LU", "NT", "NU"))


@pytest.fixture(scope="module")
def runner():
    import __graft_entry__
    __graft_entry__.build()
    return gu.Runner()


def system(rng, na, lda, uplo, diag, dtype):
    """A well-conditioned triangular A with NaN in every entry a solve must not read: the
    off-diagonal entries U[-1, 1] / na and the diagonal +-2 (or a unit diagonal), so that
    T = D + N with |D^-1 N| row sums at most 1/2 and the solution cannot grow (random
    triangular matrices with O(1) off-diagonal entries are exponentially ill conditioned and
    overflow FP32 at n ~ 1000)."""
    A = inputs.colmajor(rng, na, na, lda, np.float64)
    if na:
        M = A[: lda * na].reshape(na, lda)          # M[c, r] = A[r, c]
        M[:, :na] /= na
        for i in range(na):
            M[i, i] = 2.0 * (1 if rng.random() < 0.5 else -1)
        r, c = np.meshgrid(np.arange(na), np.arange(na), indexing="ij")
        bad = (r < c) if uplo == "L" else (r > c)
        if diag == "U":
            bad |= r == c
        M[:, :na][bad.T] = np.nan
    return A.astype(dtype)


def run(runner, side, uplo, ta, diag, m, n, alpha, A, lda, B0, ldb, policy=g.GFIP_PACK_AUTO):
    esz = A.dtype.itemsize
    dA = torch.from_numpy(A).to(runner.dev)
    Bbuf = np.concatenate([B0, np.full(gu.GUARD, np.nan, dtype=B0.dtype)])
    dB = torch.from_numpy(Bbuf).to(runner.dev)
    runner.h.set_pack_policy(policy)
    runner.h.ensure_trsm_workspace(side, uplo, ta, diag, m, n, esz)
    rc = g.gfip_trsm(esz, runner.h.h, side, uplo, ta, diag, m, n, alpha, dA.data_ptr(), lda,
                     dB.data_ptr(), ldb)
    runner.h.set_pack_policy(g.GFIP_PACK_AUTO)
    assert rc == 0, g.error_string(rc)
    torch.cuda.synchronize()
    out = dB.cpu().numpy()
    assert runner.h.status() == 0
    return out[: B0.size], out[B0.size:]


def residual_check(side, uplo, ta, diag, m, n, alpha, A, lda, B0, ldb, X, ii=None, jj=None):
    """|op(A) X - alpha B| <= c u (|op(A)||X| + |alpha B|) on all entries, or on (ii, jj)."""
    na = m if side == "L" else n
    D = np.asfortranarray(dense_op(A.astype(np.float64), lda, na, uplo, ta, diag))
    D = D.reshape(-1, order="F")
    X64 = X.astype(np.float64)
    if ii is None:
        ii, jj = (a.ravel() for a in np.meshgrid(np.arange(m), np.arange(n), indexing="ij"))
    if side == "L":
        args = ("N", "N", m, n, m, 1.0, D, na, X64, ldb, 0.0, None, m, ii, jj)
    else:
        args = ("N", "N", m, n, n, 1.0, X64, ldb, D, na, 0.0, None, m, ii, jj)
    ax = oracle.entries(*args, nthreads=8)
    mag = oracle.entries(*args, absval=True, nthreads=8)
    b = alpha * inputs.as_matrix(B0.astype(np.float64), m, n, ldb)[ii, jj]
    c = 2 * (na + 64) + 4
    u = inputs.unit_roundoff(A.dtype)
    bad = ~(np.abs(ax - b) <= c * u * (mag + np.abs(b)))
    assert not bad.any(), (side, uplo, ta, diag, m, n, int(bad.sum()))


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("side,uplo,ta,diag", COMBOS)
def test_small_and_multiblock(runner, dtype, side, uplo, ta, diag):
    rng = np.random.Generator(np.random.PCG64(21))
    for (m, n), pad, alpha in itertools.product(((1, 1), (5, 3), (33, 17), (70, 65), (130, 200)),
                                                (0, 7), (1.0, -0.75)):
        na = m if side == "L" else n
        lda, ldb = na + pad, m + pad
        A = system(rng, na, lda, uplo, diag, dtype)
        B0 = inputs.colmajor(rng, m, n, ldb, dtype)
        X, guard = run(runner, side, uplo, ta, diag, m, n, alpha, A, lda, B0, ldb)
        assert np.all(np.isnan(guard))
        if ldb > m:
            assert np.array_equal(X.reshape(n, ldb)[:, m:].view(np.uint8),
                                  B0.reshape(n, ldb)[:, m:].view(np.uint8))
        residual_check(side, uplo, ta, diag, m, n, alpha, A, lda, B0, ldb, X)
        # the oracle's solution of the same well-conditioned system
        ref = oracle.trsm_result(side, uplo, ta, diag, m, n, alpha, A.astype(np.float64), lda,
                                 B0.astype(np.float64), ldb)
        got = inputs.as_matrix(X.astype(np.float64), m, n, ldb)
        want = inputs.as_matrix(ref, m, n, ldb)
        # forward errors of a well-conditioned solve scale with the size of the solution
        # (a component near zero after cancellation has no relative accuracy of its own)
        u = inputs.unit_roundoff(A.dtype)
        scale = np.abs(want).max(axis=0 if side == "L" else 1, keepdims=True)
        assert np.all(np.abs(got - want) <= 64 * (na + 64) * u * scale), (side, uplo, ta, diag,
                                                                         m, n)


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("side,uplo,ta,diag", COMBOS)
def test_several_panels(runner, dtype, side, uplo, ta, diag):
    """Systems of 1100 unknowns: three panels of the two-level blocking (512, 512 and a
    ragged 76), forward and backward, against the residual bound and the oracle."""
    rng = np.random.Generator(np.random.PCG64(25))
    m, n = (1100, 37) if side == "L" else (37, 1100)
    na = m if side == "L" else n
    lda, ldb = na + 3, m + 5
    A = system(rng, na, lda, uplo, diag, dtype)
    B0 = inputs.colmajor(rng, m, n, ldb, dtype)
    X, guard = run(runner, side, uplo, ta, diag, m, n, -1.25, A, lda, B0, ldb)
    assert np.all(np.isnan(guard))
    residual_check(side, uplo, ta, diag, m, n, -1.25, A, lda, B0, ldb, X)
    ref = oracle.trsm_result(side, uplo, ta, diag, m, n, -1.25, A.astype(np.float64), lda,
                             B0.astype(np.float64), ldb)
    got = inputs.as_matrix(X.astype(np.float64), m, n, ldb)
    want = inputs.as_matrix(ref, m, n, ldb)
    u = inputs.unit_roundoff(A.dtype)
    scale = np.abs(want).max(axis=0 if side == "L" else 1, keepdims=True)
    assert np.all(np.abs(got - want) <= 64 * (na + 64) * u * scale)


@pytest.mark.parametrize("side,uplo,ta", list(itertools.product("LR", "LU", "NT")))
def test_integer_unit_exact_and_policies(runner, side, uplo, ta):
    """Unit systems with sparse entries in {-1, 0, 1} and small integer right-hand sides have
    integer solutions the size of the oracle's, exact in FP64; every pack policy agrees."""
    rng = np.random.Generator(np.random.PCG64(22))
    m, n = (150, 90) if side == "L" else (90, 150)
    na = m if side == "L" else n
    Ai = rng.integers(-1, 2, (na, na)) * (rng.random((na, na)) < 0.02)
    A = np.asfortranarray(Ai.astype(np.float64)).reshape(-1, order="F")
    B0 = np.asfortranarray(rng.integers(-3, 4, (m, n)).astype(np.float64)).reshape(-1, order="F")
    ref = oracle.trsm_result(side, uplo, ta, "U", m, n, 1.0, A, na, B0, m)
    if np.abs(ref).max() >= 2.0 ** 40:
        pytest.skip("solution too large for an exact comparison")
    first = None
    for policy in (g.GFIP_PACK_AUTO, g.GFIP_PACK_NONE, g.GFIP_PACK_BOTH):
        X, _ = run(runner, side, uplo, ta, "U", m, n, 1.0, A, na, B0, m, policy)
        assert np.array_equal(X, ref), policy
        if first is None:
            first = X
        assert np.array_equal(X.view(np.uint8), first.view(np.uint8))


def ieee_class(x):
    """0 NaN, 1 +inf, 2 -inf, 3 finite, element by element."""
    return np.select([np.isnan(x), np.isposinf(x), np.isneginf(x)], [0, 1, 2], 3)


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("uplo,ta", list(itertools.product("LU", "NT")))
def test_special_values_follow_ieee(runner, dtype, uplo, ta):
    """A zero on the diagonal (unknown 300 of 600), a NaN (column 0) and an infinity (column 1)
    in B: every element of X is NaN, +inf, -inf or finite exactly where the oracle's
    substitution puts one (which of the four a sum of infinities gives depends only on the
    signs of its terms, not on the order it is summed in), and the finite elements agree with
    the oracle's.  The solve meets the special values part-way through a panel, in chunks
    where every quotient is finite, in chunks where one is not, and in the short chunk that
    ends the 88-unknown second panel."""
    rng = np.random.Generator(np.random.PCG64(29))
    m, n = 600, 48
    lda, ldb = m + 3, m + 5
    A = system(rng, m, lda, uplo, "N", dtype)
    B0 = inputs.colmajor(rng, m, n, ldb, dtype)
    B0[5] = np.nan
    B0[200 + ldb] = np.inf
    # which infinity 1/0 gives follows the sign of the residual that meets the zero: with a 1
    # there instead, that residual is the solution's element, well away from zero here
    A1 = A.astype(np.float64)
    A1[300 + 300 * lda] = 1.0
    s = inputs.as_matrix(oracle.trsm_result("L", uplo, ta, "N", m, n, 1.0, A1, lda,
                                            B0.astype(np.float64), ldb), m, n, ldb)[300]
    assert np.all(np.abs(s[np.isfinite(s)]) > 1e-3)
    A[300 + 300 * lda] = 0.0
    X, guard = run(runner, "L", uplo, ta, "N", m, n, 1.0, A, lda, B0, ldb)
    assert np.all(np.isnan(guard))
    ref = oracle.trsm_result("L", uplo, ta, "N", m, n, 1.0, A.astype(np.float64), lda,
                             B0.astype(np.float64), ldb)
    got = inputs.as_matrix(X.astype(np.float64), m, n, ldb)
    want = inputs.as_matrix(ref, m, n, ldb)
    assert np.array_equal(ieee_class(got), ieee_class(want))
    fin = np.isfinite(want)
    assert fin.any() and not fin.all()
    u = inputs.unit_roundoff(dtype)
    scale = np.where(fin, np.abs(want), 0.0).max(axis=0, keepdims=True)
    err = np.abs(np.where(fin, got, 0.0) - np.where(fin, want, 0.0))
    assert np.all(err <= 64 * (m + 64) * u * scale)


def test_alpha_zero_and_codes(runner):
    m, n = 40, 30
    X, _ = run(runner, "R", "L", "T", "N", m, n, 0.0, np.full(n * n, np.nan), n,
               np.full(m * n, np.nan), m)
    assert np.all(X == 0.0)
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
        assert lib.gfip_dtrsm(runner.h.h, s_, u_, t_, d_, m_, n_, 1.0, None, lda_, None,
                              ldb_) == code


@pytest.mark.parametrize("dtype,side,uplo,ta,diag,m,n", [
    (np.float64, "L", "L", "N", "N", 4096, 2048),
    (np.float32, "R", "U", "T", "U", 2048, 4096),
])
def test_large_sampled_residual(runner, dtype, side, uplo, ta, diag, m, n):
    rng = np.random.Generator(np.random.PCG64(23))
    na = m if side == "L" else n
    A = system(rng, na, na + 7, uplo, diag, dtype)
    B0 = inputs.colmajor(rng, m, n, m + 7, dtype)
    X, guard = run(runner, side, uplo, ta, diag, m, n, 1.5, A, na + 7, B0, m + 7)
    assert np.all(np.isnan(guard))
    assert np.isfinite(inputs.as_matrix(X, m, n, m + 7)).all()
    ii, jj = inputs.sample_indices(rng, m, n, 4096, full_rows=2, full_cols=2)
    residual_check(side, uplo, ta, diag, m, n, 1.5, A, na + 7, B0, m + 7, X, ii, jj)


@pytest.mark.parametrize("solver", ["trsm", "trmm"])
def test_small_workspace_changes_nothing(runner, solver):
    """A workspace too small for the call is reported before anything is launched: B keeps
    its bytes (TRSM scales B by alpha first, so the check must come before that)."""
    rng = np.random.Generator(np.random.PCG64(24))
    m, n = 300, 200
    A = system(rng, m, m, "L", "N", np.float64)
    B0 = inputs.colmajor(rng, m, n, m + 3)
    dA = torch.from_numpy(A).to(runner.dev)
    dB = torch.from_numpy(B0.copy()).to(runner.dev)
    h = g.Handle(workspace_bytes=1 << 16)
    h.bind_stream()
    fn = g.gfip_trsm if solver == "trsm" else g.gfip_trmm
    rc = fn(8, h.h, "L", "L", "N", "N", m, n, 2.0, dA.data_ptr(), m, dB.data_ptr(), m + 3)
    assert rc == g.GFIP_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert np.array_equal(dB.cpu().numpy().view(np.uint8), B0.view(np.uint8))
