"""The CUDA path against the same external pins as the oracle, FP64 through the C ABI.

GEMM (tests/oracle_pins.py), for the fused routine (both packers), the direct and the
pack-then-compute variants: hand-derived textbook products and integer products bit-exact,
identity, permutation and rank-1 operands exact, numpy's float64 matmul within the bound,
exact rational arithmetic within (k + 3) u on tiny shapes, and the reference-BLAS rules
(argument codes, quick returns, operands that must not be read, gap rows of C untouched).

SYRK, TRMM and TRSM (the pins of tests/test_oracle_{syrk,trmm,trsm}.py): exact rational
brute force on tiny shapes within the oracle's bounds, hand-worked products, integer
operands exact, TRSM undoing TRMM, and the BLAS rules.  The oracle pins that compare
bit for bit with the GEMM oracle's rounding sequence (no FMA) do not apply to the GPU and
are not run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_08417_gb300 import gemmfip as g  # noqa: E402
from tests import gpu_util as gu  # noqa: E402
from tests import oracle_pins as pins  # noqa: E402
from tests import test_oracle_syrk as syrk_pins  # noqa: E402
from tests import test_oracle_trmm as trmm_pins  # noqa: E402
from tests import test_oracle_trsm as trsm_pins  # noqa: E402


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


def _up(runner, X):
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.float64)).to(runner.dev)


def _ptr(t):
    return t.data_ptr() if t.numel() else 0


def cuda_syrk(runner):
    def syrk(uplo, trans, n, k, alpha, A, lda, beta, C, ldc):
        dA, dC = _up(runner, A), _up(runner, C)
        runner.h.ensure_syrk_workspace(uplo, trans, n, k, 8)
        rc = g.gfip_syrk(8, runner.h.h, uplo, trans, n, k, alpha, _ptr(dA), lda, beta,
                         _ptr(dC), ldc)
        torch.cuda.synchronize()
        C[...] = dC.cpu().numpy()
        assert runner.h.status() == 0
        return rc
    return syrk


def cuda_triangular(runner, solve):
    """gfip_dtrsm (solve) or gfip_dtrmm with the oracle's signature; B in place."""
    def op(side, uplo, ta, diag, m, n, alpha, A, lda, B, ldb):
        dA, dB = _up(runner, A), _up(runner, B)
        if solve:
            runner.h.ensure_trsm_workspace(side, uplo, ta, diag, m, n, 8)
        else:
            runner.h.ensure_trmm_workspace(side, uplo, ta, diag, m, n, 8)
        fn = g.gfip_trsm if solve else g.gfip_trmm
        rc = fn(8, runner.h.h, side, uplo, ta, diag, m, n, alpha, _ptr(dA), lda, _ptr(dB), ldb)
        torch.cuda.synchronize()
        B[...] = dB.cpu().numpy()
        assert runner.h.status() == 0
        return rc
    return op


@pytest.mark.parametrize("pin", [syrk_pins.pin_bruteforce, syrk_pins.pin_handworked,
                                 syrk_pins.pin_integer_exact, syrk_pins.pin_blas_rules],
                         ids=lambda f: f.__name__)
def test_cuda_syrk_passes_oracle_pins(runner, pin):
    pin(cuda_syrk(runner))


@pytest.mark.parametrize("pin", [trmm_pins.pin_bruteforce, trmm_pins.pin_handworked,
                                 trmm_pins.pin_integer_exact, trmm_pins.pin_blas_rules],
                         ids=lambda f: f.__name__)
def test_cuda_trmm_passes_oracle_pins(runner, pin):
    pin(cuda_triangular(runner, solve=False))


@pytest.mark.parametrize("pin", trsm_pins.TRSM_PINS, ids=lambda f: f.__name__)
def test_cuda_trsm_passes_oracle_pins(runner, pin):
    pin(cuda_triangular(runner, solve=True))

