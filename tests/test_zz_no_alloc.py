"""The allocation-free entry point gfip_dgemm_noalloc, through the C ABI.

It serves callers that cannot allocate device memory or pass a workspace (code behind the
plain BLAS dgemm interface, applications that own all device memory, code where cudaMalloc is
not allowed): its scratch is a fixed static device array inside the library.  This file is
named so that pytest collects it last; it builds the library itself, so it also runs alone
in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_08417_gb300 import gemmfip as g  # noqa: E402
from paper_2302_08417_gb300 import inputs  # noqa: E402
from tests import gpu_util as gu  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    return torch.device("cuda", 0)


def _run_both(p, dev, stream):
    A = torch.from_numpy(p.A).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    C_ref = torch.from_numpy(p.C0).to(dev)
    C_new = torch.from_numpy(p.C0).to(dev)
    h = g.Handle()
    h.bind_stream()
    h.ensure_workspace(p.transa, p.transb, p.m, p.n, p.k, 8)
    rc = g.gfip_dgemm(h.h, p.transa, p.transb, p.m, p.n, p.k, p.alpha, A.data_ptr(), p.lda,
                      B.data_ptr(), p.ldb, p.beta, C_ref.data_ptr(), p.ldc)
    assert rc == 0, g.error_string(rc)
    rc = g.gfip_dgemm_noalloc(p.transa, p.transb, p.m, p.n, p.k, p.alpha, A.data_ptr(), p.lda,
                              B.data_ptr(), p.ldb, p.beta, C_new.data_ptr(), p.ldc, stream)
    assert rc == 0, g.error_string(rc)
    torch.cuda.synchronize()
    return C_ref.cpu().numpy(), C_new.cpu().numpy()


def test_noalloc_matches_gfip_dgemm_two_calls_in_a_row(dev):
    """Same kernel and same launch plan as gfip_dgemm, so the same result bits over the whole
    ldc x n buffer (gap rows included); and within the tolerance of the other parity tests,
    2 max(k, 2) u (|alpha||op(A)||op(B)| + |beta||C0|), against the oracle."""
    stream = torch.cuda.current_stream().cuda_stream
    problems = [
        inputs.problem(501, "N", "T", 700, 650, 300, 1.0, 0.5, 7, 7, 7),
        inputs.problem(502, "T", "N", 1000, 333, 999, -1.25, 0.0, 0, 7, 3),
    ]
    for p in problems:   # two calls in a row, different shapes: the shared array is reused
        ref, new = _run_both(p, dev, stream)
        assert np.array_equal(new.view(np.uint64), ref.view(np.uint64))
        want, absterm = gu.reference(p)
        gu.assert_close(p, new, want, absterm, label="noalloc")
        # rows m..ldc-1 of C are never written
        if p.ldc > p.m:
            gap = new.reshape(p.n, p.ldc)[:, p.m:]
            assert np.all(np.isnan(gap))


def test_noalloc_rejects_problems_beyond_its_scratch(dev):
    m = n = k = 4096
    # real buffers of the full size, so the call would be valid if it were not rejected
    A = torch.zeros(m * k, dtype=torch.float64, device=dev)
    B = torch.zeros(k * n, dtype=torch.float64, device=dev)
    C = torch.full((m * n,), 3.0, dtype=torch.float64, device=dev)
    rc = g.gfip_dgemm_noalloc("N", "N", m, n, k, 1.0, A.data_ptr(), m, B.data_ptr(), k, 0.0,
                              C.data_ptr(), m, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == g.GFIP_ERR_SCRATCH_LIMIT
    assert bool((C == 3.0).all()), "a rejected call must leave C untouched"
    assert "scratch" in g.error_string(rc)
