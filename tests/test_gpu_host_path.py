"""The end-to-end path of the public ``gemm()``: host operands in, host result out, through
the C ABI.  The pipelined form (column blocks of C uploaded, computed and downloaded on
three streams) and the single-call form against the oracle within the GEMM bound, on
padded leading dimensions, both transa, beta zero and non-zero, pinned and pageable host
memory; rows m..ldc-1 of the host C keep their bytes."""
import itertools

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
def handle():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    return g.Handle()


def host_view(flat, rows, cols, ld, pinned):
    """A column-major rows x cols view with leading dimension ld of a host copy of flat."""
    t = torch.from_numpy(flat.copy())
    if pinned:
        t = t.pin_memory()
    return torch.as_strided(t, (rows, cols), (1, ld)), t


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("transa,transb,beta,pinned,block", [
    ("N", "N", 0.5, True, 64),     # pipelined, 4 blocks of ragged width
    ("T", "N", 0.0, True, 64),     # pipelined, beta 0: C not uploaded when ldc == m
    ("N", "N", 0.0, False, 100),   # pipelined from pageable memory, 3 blocks
    ("N", "T", 0.5, True, 64),     # op(B) = B^T: one call
    ("T", "T", 1.0, False, 1024),  # fewer columns than two blocks: one call
])
def test_host_path_against_oracle(handle, monkeypatch, dtype, transa, transb, beta, pinned,
                                  block):
    monkeypatch.setattr(g, "HOST_BLOCK_COLS", block)
    for seed, (pad_c, (m, n, k)) in enumerate(itertools.product(
            (0, 5), ((300, 290, 170), (129, 333, 64)))):
        p = inputs.problem(40 + seed, transa, transb, m, n, k, alpha=-1.25, beta=beta,
                           pad_a=7, pad_b=3, pad_c=pad_c, dtype=dtype)
        A, _ = host_view(p.A, p.rows_a, p.cols_a, p.lda, pinned)
        B, _ = host_view(p.B, p.rows_b, p.cols_b, p.ldb, pinned)
        C, Cbuf = host_view(p.C0, p.m, p.n, p.ldc, pinned)
        out = g.gemm(A, B, C, p.alpha, p.beta, transa, transb, handle=handle)
        assert out is C
        got = Cbuf.numpy()
        gu.assert_close(p, got, label="host path")
        if p.ldc > p.m:
            gap = got.reshape(p.n, p.ldc)[:, p.m:]
            want = p.C0[: p.n * p.ldc].reshape(p.n, p.ldc)[:, p.m:]
            assert np.array_equal(gap.view(np.uint8), want.view(np.uint8))
        assert handle.status() == 0


def test_host_path_allocates_c(handle, monkeypatch):
    """C = None: the result is a new pinned column-major host tensor."""
    monkeypatch.setattr(g, "HOST_BLOCK_COLS", 64)
    p = inputs.problem(50, "N", "N", 200, 260, 90, alpha=1.0, beta=0.0)
    A, _ = host_view(p.A, p.m, p.k, p.lda, True)
    B, _ = host_view(p.B, p.k, p.n, p.ldb, True)
    C = g.gemm(A, B, None, p.alpha, 0.0)
    assert not C.is_cuda and C.is_pinned() and C.stride() == (1, p.m)
    flat = torch.as_strided(C, (p.m * p.n,), (1,)).numpy().copy()
    gu.assert_close(p, flat, label="allocated C")
