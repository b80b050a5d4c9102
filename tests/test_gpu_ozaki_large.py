"""FP64 emulated on the tensor cores (gfip_dgemm_ozaki) at the sizes of its workload:
m = n = k in {2048, 4096, 8192, 16384}, transa = transb = 'N', entries uniform[-1, 1] and
log-uniform magnitudes in [1e-4, 1e4] with random sign, 3, 5, 7 and 9 digits.

At 2048 the whole result is compared with the oracle; above it, sampled entries are: 4096
random (i, j) plus 8 whole rows and 8 whole columns, each computed by the oracle one by one.
Every entry must lie within the splitting bound of test_gpu_ozaki.py,
    |alpha| k 2^(e_i+f_j) (2^(-6S) (S+2) + 16 (P*chunks + 2) u) + 2u |beta C0|.
These launches hold far more 128 x 128 tiles (256 at 2048, 16384 at 16384) than the GPU has
SMs, so every SM allocates, uses and releases tensor memory many times within one launch,
which the small shapes of test_gpu_ozaki.py never do."""
import os

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
from tests.test_gpu_ozaki import exponents, split_bound  # noqa: E402

U = 2.0 ** -53
THREADS = os.cpu_count() or 1
SLICES = (3, 5, 7, 9)


@pytest.fixture(scope="module")
def runner():
    import __graft_entry__
    __graft_entry__.build()
    return gu.Runner()


def sampled_bound(p: inputs.Problem, slices: int, ii, jj):
    """The splitting bound at the entries (ii[t], jj[t])."""
    ea, eb = exponents(p)
    pairs = slices * (slices + 1) // 2
    chunks = max(1, -(-p.k // 16384))
    rel = 2.0 ** (-6 * slices) * (slices + 2) + 16 * (pairs * chunks + 2) * U
    tol = abs(p.alpha) * p.k * np.exp2(ea[ii] + eb[jj]) * rel
    if p.beta != 0:
        c0 = inputs.as_matrix(p.C0, p.m, p.n, p.ldc)[ii, jj]
        tol = tol + 2 * U * np.abs(p.beta * c0)
    return tol


class Device:
    """The operands of one problem on the GPU, and one emulated call at a time."""

    def __init__(self, runner, p: inputs.Problem):
        self.runner, self.p = runner, p
        self.A = torch.from_numpy(p.A).to(runner.dev)
        self.B = torch.from_numpy(p.B).to(runner.dev)
        self.C0 = torch.from_numpy(p.C0).to(runner.dev)
        self.C = torch.empty_like(self.C0)

    def run(self, slices: int) -> np.ndarray:
        p, h = self.p, self.runner.h
        self.C.copy_(self.C0)
        h.ensure_ozaki_workspace(p.m, p.n, p.k, slices)
        rc = g.gfip_dgemm_ozaki(h.h, p.transa, p.transb, p.m, p.n, p.k, p.alpha,
                                self.A.data_ptr(), p.lda, self.B.data_ptr(), p.ldb, p.beta,
                                self.C.data_ptr(), p.ldc, slices)
        assert rc == 0, g.error_string(rc)
        torch.cuda.synchronize()
        assert h.status() == 0
        return self.C.cpu().numpy()


def check_gap(p: inputs.Problem, got_flat):
    if p.ldc > p.m:
        gap = got_flat.reshape(p.n, p.ldc)[:, p.m:]
        assert np.all(np.isnan(gap)), "rows m..ldc-1 of C written"


@pytest.mark.parametrize("dist", ["uniform", "logmag"])
def test_2048_whole_result_within_splitting_bound(runner, dist):
    n = 2048
    p = inputs.problem(2048 + (dist == "logmag"), "N", "N", n, n, n, 1.0, 0.5, 7, 7, 7,
                       dist=dist)
    ref, _ = gu.reference(p)
    want = inputs.as_matrix(ref, n, n, p.ldc)
    d = Device(runner, p)
    for s in SLICES:
        got = d.run(s)
        check_gap(p, got)
        err = np.abs(inputs.as_matrix(got, n, n, p.ldc) - want)
        tol = split_bound(p, s)
        assert np.all(err <= tol), (dist, s, float((err / tol).max()))


CASES = [(4096, d, SLICES) for d in ("uniform", "logmag")] + \
        [(8192, d, SLICES) for d in ("uniform", "logmag")] + \
        [(16384, "uniform", (7,))]


@pytest.mark.parametrize("n,dist,slices", CASES,
                         ids=[f"{c[0]}-{c[1]}-S{'_'.join(map(str, c[2]))}" for c in CASES])
def test_sampled_entries_within_splitting_bound(runner, n, dist, slices):
    p = inputs.problem(n + 3 * (dist == "logmag"), "N", "N", n, n, n, 1.0, 0.5, 7, 7, 7,
                       dist=dist)
    rng = np.random.Generator(np.random.PCG64(n + 17))
    ii, jj = inputs.sample_indices(rng, n, n, 4096, full_rows=8, full_cols=8)
    args = (p.transa, p.transb, p.m, p.n, p.k, p.alpha, p.A, p.lda, p.B, p.ldb, p.beta, p.C0,
            p.ldc, ii, jj)
    want = oracle.entries(*args, nthreads=THREADS)
    d = Device(runner, p)
    for s in slices:
        got_flat = d.run(s)
        check_gap(p, got_flat)
        got = inputs.as_matrix(got_flat, n, n, p.ldc)[ii, jj]
        err = np.abs(got - want)
        tol = sampled_bound(p, s, ii, jj)
        bad = ~(err <= tol)
        assert not bad.any(), (
            f"{n} {dist} S={s}: {int(bad.sum())} of {ii.size} sampled entries out of the "
            f"splitting bound; worst ratio {float((err / tol).max()):.3g}")
