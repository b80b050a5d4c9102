"""FP64 GEMM emulated with BF16 digit products on the tensor cores (gfip_dgemm_ozaki),
through the C ABI, against the FP64 oracle.

* Small-integer operands split into digits exactly, so the emulated product equals the
  oracle bit for bit for every digit count: this pins the tensor-core path itself (tile
  layout, descriptors, accumulator read-out, recombination).
* General data: the error is within the splitting bound
      |alpha| k 2^(e_i+f_j) (2^(-6S) (S+2) + 16 (P*chunks + 2) u) + 2u |beta C0|,
  2^e_i, 2^f_j the powers of two above the largest magnitude in row i of op(A) and column j
  of op(B), P = S(S+1)/2 digit pairs, chunks = ceil(k / 16384), u = 2^-53.  (Elements are
  scaled below 1/2, so digit truncation and the dropped pairs s + t > S + 1 cost at most
  2^(e_i+f_j+2) 2^(-6S) ((1 + (S-1)/4) / 2) per product, which (S+2) 2^(-6S) 2^(e_i+f_j)
  covers, and the FP64 recombination adds one rounding per unit of terms below
  4 k 2^(e_i+f_j).)
"""
import itertools
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_08417_gb300 import gemmfip as g  # noqa: E402
from paper_2302_08417_gb300 import inputs  # noqa: E402
from tests import gpu_util as gu  # noqa: E402

U = 2.0 ** -53


@pytest.fixture(scope="module")
def runner():
    import __graft_entry__
    __graft_entry__.build()
    return gu.Runner()


def run_ozaki(runner, p: inputs.Problem, slices: int, C_init=None):
    A = torch.from_numpy(p.A).to(runner.dev)
    B = torch.from_numpy(p.B).to(runner.dev)
    c0 = p.C0 if C_init is None else C_init
    Cbuf = np.concatenate([c0, np.full(gu.GUARD, np.nan)])
    C = torch.from_numpy(Cbuf).to(runner.dev)
    runner.h.ensure_ozaki_workspace(p.m, p.n, p.k, slices)
    rc = g.gfip_dgemm_ozaki(runner.h.h, p.transa, p.transb, p.m, p.n, p.k, p.alpha,
                            A.data_ptr(), p.lda, B.data_ptr(), p.ldb, p.beta, C.data_ptr(),
                            p.ldc, slices)
    assert rc == 0, g.error_string(rc)
    torch.cuda.synchronize()
    out = C.cpu().numpy()
    assert runner.h.status() == 0
    return out[: c0.size], out[c0.size:]


def exponents(p: inputs.Problem):
    """e_i and f_j: smallest powers of two strictly above each row / column maximum."""
    opa = inputs.as_matrix(p.A, p.rows_a, p.cols_a, p.lda)
    opa = opa if inputs.is_notrans(p.transa) else opa.T
    opb = inputs.as_matrix(p.B, p.rows_b, p.cols_b, p.ldb)
    opb = opb if inputs.is_notrans(p.transb) else opb.T
    ma = np.abs(opa).max(axis=1) if p.k else np.zeros(p.m)
    mb = np.abs(opb).max(axis=0) if p.k else np.zeros(p.n)
    ea = np.array([math.frexp(x)[1] if x > 0 else 0 for x in ma], dtype=np.float64)
    eb = np.array([math.frexp(x)[1] if x > 0 else 0 for x in mb], dtype=np.float64)
    return ea, eb


def split_bound(p: inputs.Problem, slices: int):
    ea, eb = exponents(p)
    pairs = slices * (slices + 1) // 2
    chunks = max(1, -(-p.k // 16384))
    scale = np.exp2(ea[:, None] + eb[None, :])
    rel = 2.0 ** (-6 * slices) * (slices + 2) + 16 * (pairs * chunks + 2) * U
    tol = abs(p.alpha) * p.k * scale * rel
    if p.beta != 0:
        tol = tol + 2 * U * np.abs(p.beta * inputs.as_matrix(p.C0, p.m, p.n, p.ldc))
    return tol


@pytest.mark.parametrize("slices", [1, 2, 3])
@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
def test_integer_operands_bit_exact(runner, ta, tb, slices):
    for (m, n, k), (alpha, beta) in itertools.product(
            [(130, 129, 70), (256, 128, 64), (1, 300, 17000), (200, 1, 33)],
            [(1.0, 0.0), (2.0, 0.5)]):
        p = inputs.problem(61, ta, tb, m, n, k, alpha, beta, 3, 5, 7, dist="int", int_lim=4)
        got, guard = run_ozaki(runner, p, slices)
        ref, _ = gu.reference(p)
        a = inputs.as_matrix(got, m, n, p.ldc)
        b = inputs.as_matrix(ref, m, n, p.ldc)
        assert np.array_equal(a, b), (ta, tb, m, n, k, slices, np.abs(a - b).max())
        gu.assert_gap_untouched(p, got, guard)


@pytest.mark.parametrize("dist", ["uniform", "logmag"])
@pytest.mark.parametrize("slices", [3, 5, 7, 9])
def test_error_within_splitting_bound(runner, dist, slices):
    for (ta, tb), (m, n, k) in itertools.product(
            [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")],
            [(300, 260, 200), (33, 65, 17000)]):
        p = inputs.problem(71 + slices, ta, tb, m, n, k, -1.25, 0.5, 7, 0, 7, dist=dist)
        got, guard = run_ozaki(runner, p, slices)
        ref, _ = gu.reference(p)
        err = np.abs(inputs.as_matrix(got, m, n, p.ldc) - inputs.as_matrix(ref, m, n, p.ldc))
        tol = split_bound(p, slices)
        assert np.all(err <= tol), (ta, tb, m, n, k, slices, (err / tol).max())
        gu.assert_gap_untouched(p, got, guard)


def test_nine_digits_reach_fp64_accuracy(runner):
    """uniform[-1,1] data: 9 digits (54 bits) are within the FP64 GEMM bound of the tests."""
    p = inputs.problem(81, "N", "N", 512, 512, 512, 1.0, 0.5, 7, 7, 7)
    got, _ = run_ozaki(runner, p, 9)
    gu.assert_close(p, got, label="ozaki9")


def test_beta_zero_does_not_read_c(runner):
    p = inputs.problem(91, "T", "N", 150, 140, 90, 1.0, 0.0, 1, 1, 1)
    got, _ = run_ozaki(runner, p, 4, C_init=np.full_like(p.C0, np.nan))
    assert not np.isnan(inputs.as_matrix(got, p.m, p.n, p.ldc)).any()


def test_bad_slice_count_rejected(runner):
    for s in (0, 11):
        rc = g.gfip_dgemm_ozaki(runner.h.h, "N", "N", 4, 4, 4, 1.0, 16, 4, 16, 4, 0.0, 16, 4, s)
        assert rc == g.GFIP_ERR_ARG


def test_wait_timeout_reports_status_and_recovers(runner):
    """The failure path: with the test hook on, the first CTA withholds one operand copy and
    its bounded wait runs out after 20 ms.  The call raises GFIP_STATUS_MMA_TIMEOUT, leaves
    that CTA's 128 x 128 tile of C unwritten, computes every other tile, and the context
    stays usable: the next call, hook off, is exact again."""
    p = inputs.problem(95, "N", "N", 300, 260, 200, 1.0, 0.0, 3, 3, 3, dist="int", int_lim=4)
    ref, _ = gu.reference(p)
    want = inputs.as_matrix(ref, p.m, p.n, p.ldc)
    marker = np.where(np.isnan(p.C0), p.C0, 12345.0)     # beta == 0: C is never read
    A = torch.from_numpy(p.A).to(runner.dev)
    B = torch.from_numpy(p.B).to(runner.dev)
    C = torch.from_numpy(marker.copy()).to(runner.dev)
    runner.h.ensure_ozaki_workspace(p.m, p.n, p.k, 3)
    assert runner.h.status() == 0
    assert g.gfip_debug_ozaki_timeout(runner.h.h, True, 20_000_000) == 0
    try:
        rc = g.gfip_dgemm_ozaki(runner.h.h, "N", "N", p.m, p.n, p.k, 1.0, A.data_ptr(), p.lda,
                                B.data_ptr(), p.ldb, 0.0, C.data_ptr(), p.ldc, 3)
        assert rc == 0
        torch.cuda.synchronize()
    finally:
        assert g.gfip_debug_ozaki_timeout(runner.h.h, False, 0) == 0
    assert runner.h.status() & g.GFIP_STATUS_MMA_TIMEOUT
    got = inputs.as_matrix(C.cpu().numpy(), p.m, p.n, p.ldc)
    assert np.all(got[:128, :128] == 12345.0)            # the withholding CTA's tile
    rest = np.ones_like(got, dtype=bool)
    rest[:128, :128] = False
    assert np.array_equal(got[rest], want[rest])
    # recovery: same call, hook off
    C.copy_(torch.from_numpy(marker.copy()))
    rc = g.gfip_dgemm_ozaki(runner.h.h, "N", "N", p.m, p.n, p.k, 1.0, A.data_ptr(), p.lda,
                            B.data_ptr(), p.ldb, 0.0, C.data_ptr(), p.ldc, 3)
    assert rc == 0
    torch.cuda.synchronize()
    assert runner.h.status() == 0
    assert np.array_equal(inputs.as_matrix(C.cpu().numpy(), p.m, p.n, p.ldc), want)
