"""The CUDA path against the same external pins as the oracle (tests/oracle_pins.py):
hand-derived textbook products and integer products bit-exact, identity, permutation and
rank-1 operands exact, numpy's float64 matmul within the bound, exact rational arithmetic
within (k + 3) u on tiny shapes, and the reference-BLAS rules (argument codes, quick returns,
operands that must not be read, gap rows of C untouched).  FP64 through the C ABI, for the
fused routine (both packers), the direct and the pack-then-compute variants."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_08417_gb300 import gemmfip as g  # noqa: E402
from tests import gpu_util as gu  # noqa: E402
from tests import oracle_pins as pins  # noqa: E402


@pytest.fixture(scope="module")
def runner():
    import __graft_entry__
    __graft_entry__.build()
    return gu.Runner()


def cuda_gemm(runner, variant, policy, packer):
    """A callable with the oracle's signature that runs one FP64 GEMM on the GPU: the
    operand buffers are copied up as they are, C is computed in place and copied back."""
    name = g.ENTRY[(variant, 8)]

    def gemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, nthreads=1):
        dA = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float64)).to(runner.dev)
        dB = torch.from_numpy(np.ascontiguousarray(B, dtype=np.float64)).to(runner.dev)
        dC = torch.from_numpy(np.ascontiguousarray(C, dtype=np.float64)).to(runner.dev)
        runner.h.set_pack_policy(policy)
        runner.h.set_packer(packer)
        try:
            runner.h.ensure_workspace(transa, transb, m, n, k, 8)
            rc = g._gemm_call(name, runner.h.h, transa, transb, m, n, k, alpha,
                              dA.data_ptr() if dA.numel() else 0, lda,
                              dB.data_ptr() if dB.numel() else 0, ldb, beta,
                              dC.data_ptr() if dC.numel() else 0, ldc)
            torch.cuda.synchronize()
        finally:
            runner.h.set_pack_policy(g.GFIP_PACK_AUTO)
            runner.h.set_packer(g.GFIP_PACKER_AUTO)
        C[...] = dC.cpu().numpy()
        assert runner.h.status() == 0
        return rc
    return gemm


CONFIGS = {
    "fused": ("fused", g.GFIP_PACK_AUTO, g.GFIP_PACKER_AUTO),
    "fused_shared_both": ("fused", g.GFIP_PACK_BOTH, g.GFIP_PACKER_SHARED),
    "fused_line_both": ("fused", g.GFIP_PACK_BOTH, g.GFIP_PACKER_LINE),
    "direct": ("direct", g.GFIP_PACK_AUTO, g.GFIP_PACKER_AUTO),
    "pack_then_compute": ("pack_then_compute", g.GFIP_PACK_AUTO, g.GFIP_PACKER_AUTO),
}
CHEAP = [pins.pin_golden, pins.pin_closed_forms, pins.pin_integer_exact,
         pins.pin_numpy_matmul, pins.pin_blas_rules]


@pytest.mark.parametrize("config", sorted(CONFIGS))
@pytest.mark.parametrize("pin", CHEAP, ids=lambda f: f.__name__)
def test_cuda_path_passes_oracle_pins(runner, config, pin):
    pin(cuda_gemm(runner, *CONFIGS[config]))


@pytest.mark.parametrize("config", ["fused", "fused_shared_both"])
def test_cuda_path_exact_rational_bound(runner, config):
    pins.pin_fraction_bruteforce(cuda_gemm(runner, *CONFIGS[config]), sizes=(0, 1, 2, 5),
                                 trans="NTc")
