"""The CPU oracle against its pins (no GPU needed)."""
import numpy as np
import pytest

import oracle
from paper_2302_08417_gb300 import inputs
from tests import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    pin(oracle.gemm)


def test_entries_match_full_product_bitwise():
    """The sampled-entry routine reproduces the full routine's bits (same summation order),
    and its absval mode equals |alpha||A||B| + |beta||C0| from numpy within rounding."""
    for ta, tb in (("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")):
        p = inputs.problem(5, ta, tb, 33, 17, 41, -1.25, 0.5, 7, 3, 7)
        C = oracle.gemm_result(ta, tb, p.m, p.n, p.k, p.alpha, p.A, p.lda, p.B, p.ldb,
                               p.beta, p.C0, p.ldc)
        rng = np.random.Generator(np.random.PCG64(1))
        ii, jj = inputs.sample_indices(rng, p.m, p.n, 50, full_rows=2, full_cols=2)
        e = oracle.entries(ta, tb, p.m, p.n, p.k, p.alpha, p.A, p.lda, p.B, p.ldb, p.beta,
                           p.C0, p.ldc, ii, jj)
        full = inputs.as_matrix(C, p.m, p.n, p.ldc)
        assert np.array_equal(e, full[ii, jj])
        ab = oracle.abs_bound(ta, tb, p.m, p.n, p.k, p.alpha, p.A, p.lda, p.B, p.ldb,
                              p.beta, p.C0, p.ldc)
        opa = inputs.as_matrix(p.A, p.rows_a, p.cols_a, p.lda)
        opa = opa if ta == "N" else opa.T
        opb = inputs.as_matrix(p.B, p.rows_b, p.cols_b, p.ldb)
        opb = opb if tb == "N" else opb.T
        want = 1.25 * (np.abs(opa) @ np.abs(opb)) + 0.5 * np.abs(
            inputs.as_matrix(p.C0, p.m, p.n, p.ldc))
        assert np.allclose(ab, want, rtol=1e-13, atol=0)


def test_thread_count_does_not_change_bits():
    p = inputs.problem(9, "T", "N", 70, 90, 50, 1.0, 0.5, 7, 7, 7)
    c1 = oracle.gemm_result("T", "N", p.m, p.n, p.k, 1.0, p.A, p.lda, p.B, p.ldb, 0.5, p.C0,
                            p.ldc, nthreads=1)
    c4 = oracle.gemm_result("T", "N", p.m, p.n, p.k, 1.0, p.A, p.lda, p.B, p.ldb, 0.5, p.C0,
                            p.ldc, nthreads=4)
    assert np.array_equal(c1, c4, equal_nan=True)


def test_entries_rejects_out_of_range_index():
    p = inputs.problem(1, "N", "N", 4, 4, 4)
    with pytest.raises(ValueError):
        oracle.entries("N", "N", 4, 4, 4, 1.0, p.A, p.lda, p.B, p.ldb, 0.0, p.C0, p.ldc,
                       [4], [0])
