"""GB300 (sm_103a) fused-in-packing GEMM (GEMMFIP, arXiv 2302.08417) for FP64 and FP32.

``C := alpha*op(A)*op(B) + beta*C`` on BLAS column-major strided operands, computed by the
CUDA library ``_build/libgemmfip.so`` behind the C ABI of ``include/gemmfip.h``.  The
binding in :mod:`.gemmfip` mirrors that ABI; :func:`gemm` is the PyTorch-facing call and
:mod:`.autograd` its differentiable form.
"""
from .gemmfip import (  # noqa: F401
    GemmError, Handle, gemm, load, error_string, default_handle,
    GFIP_PACK_AUTO, GFIP_PACK_NONE, GFIP_PACK_A, GFIP_PACK_B, GFIP_PACK_BOTH,
)
