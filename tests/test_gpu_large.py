"""Full-size parity: the largest squares of the 16..16384 spectrum and the skinny shapes,
through the C ABI, in the launch configuration the benchmark times.

The oracle computes sampled entries one by one: 4096 random (i, j) plus 8 whole rows and
8 whole columns of C, each against 2 max(k, 2) u (|alpha||op(A)||op(B)| + |beta||C0|).
The rows m..ldc-1 of C and a guard after it must keep their NaN sentinels, and the variants
(fused, direct, pack-then-compute) must agree bit for bit, since they share one schedule."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2302_08417_gb300 import inputs  # noqa: E402
from tests import gpu_util as gu  # noqa: E402

THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def runner():
    import __graft_entry__
    __graft_entry__.build()
    return gu.Runner()


def sampled_check(p: inputs.Problem, got_flat, seed: int, label: str):
    rng = np.random.Generator(np.random.PCG64(seed))
    ii, jj = inputs.sample_indices(rng, p.m, p.n, 4096, full_rows=8, full_cols=8)
    A, B, C0 = (x.astype(np.float64, copy=False) for x in (p.A, p.B, p.C0))
    args = (p.transa, p.transb, p.m, p.n, p.k, p.alpha, A, p.lda, B, p.ldb, p.beta, C0,
            p.ldc, ii, jj)
    ref = oracle.entries(*args, nthreads=THREADS)
    ab = oracle.entries(*args, absval=True, nthreads=THREADS)
    got = inputs.as_matrix(got_flat, p.m, p.n, p.ldc)[ii, jj].astype(np.float64)
    tol = 2.0 * max(p.k, 2) * inputs.unit_roundoff(p.A.dtype) * ab
    err = np.abs(got - ref)
    bad = ~(err <= tol)
    assert not bad.any(), (
        f"{label}: {int(bad.sum())} of {ii.size} sampled entries out of bound; first at "
        f"({ii[bad][0]}, {jj[bad][0]}): got {got[bad][0]!r} want {ref[bad][0]!r}")


CASES = [
    # (dtype, transa, transb, m, n, k, pad, beta, variants)
    (np.float64, "N", "N", 8192, 8192, 8192, 7, 0.5, ("fused", "direct", "pack_then_compute")),
    (np.float32, "T", "T", 8192, 8192, 8192, 0, 0.0, ("fused", "direct", "pack_then_compute")),
    (np.float32, "N", "N", 8192, 8192, 8192, 7, 0.5, ("fused", "pack_then_compute")),
    (np.float64, "N", "T", 8192, 8192, 64, 7, 0.5, ("fused", "direct", "pack_then_compute")),
    (np.float64, "T", "N", 64, 8192, 8192, 7, 0.0, ("fused", "direct", "pack_then_compute")),
    (np.float64, "N", "N", 8192, 64, 8192, 0, 0.5, ("fused", "direct", "pack_then_compute")),
    (np.float32, "T", "T", 8192, 8192, 64, 0, 0.5, ("fused", "direct", "pack_then_compute")),
    (np.float32, "N", "T", 64, 8192, 8192, 7, 0.5, ("fused", "direct", "pack_then_compute")),
    (np.float32, "T", "N", 8192, 64, 8192, 7, 0.0, ("fused", "direct", "pack_then_compute")),
]


@pytest.mark.parametrize("dtype,ta,tb,m,n,k,pad,beta,variants", CASES,
                         ids=[f"{np.dtype(c[0]).name}-{c[1]}{c[2]}-{c[3]}x{c[4]}x{c[5]}-pad{c[6]}"
                              for c in CASES])
def test_large_sampled(runner, dtype, ta, tb, m, n, k, pad, beta, variants):
    p = inputs.problem(m + 3 * n + 7 * k + pad, ta, tb, m, n, k, 1.0, beta, pad, pad, pad,
                       dtype=dtype)
    A = torch.from_numpy(p.A).to(runner.dev)
    B = torch.from_numpy(p.B).to(runner.dev)
    first = None
    for variant in variants:
        got, guard = runner.run(p, variant, A_dev=A, B_dev=B)
        gu.assert_gap_untouched(p, got, guard)
        if first is None:
            first = got
            sampled_check(p, got, seed=m + n + k, label=variant)
        else:
            assert np.array_equal(got.view(np.uint8), first.view(np.uint8)), variant
    assert runner.h.status() == 0


def test_16384_fp64_fused_and_direct(runner):
    """The largest size of the spectrum, FP64 N/N with ld = m + 7 (about 7 s per call)."""
    n = 16384
    p = inputs.problem(16384, "N", "N", n, n, n, 1.0, 0.5, 7, 7, 7)
    A = torch.from_numpy(p.A).to(runner.dev)
    B = torch.from_numpy(p.B).to(runner.dev)
    got, guard = runner.run(p, "fused", A_dev=A, B_dev=B)
    gu.assert_gap_untouched(p, got, guard)
    sampled_check(p, got, seed=5, label="fused 16384")
    again, _ = runner.run(p, "direct", A_dev=A, B_dev=B)
    assert np.array_equal(again.view(np.uint8), got.view(np.uint8))
    assert runner.h.status() == 0
