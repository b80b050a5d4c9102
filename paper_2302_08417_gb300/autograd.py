"""Differentiable GEMM: C = alpha * op(A) * op(B), with both gradients computed by the
fused-in-packing kernel on transposed operand strides.

Backward of C = alpha * op(A) op(B) for an upstream gradient dC (m x n):

    d op(A) = alpha * dC * op(B)^T        (m x k)
    d op(B) = alpha * op(A)^T * dC        (k x n)

mapped back through op(): when A is stored transposed (transa = 'T', A is k x m), the stored
gradient is dA = (d op(A))^T = alpha * op(B) * dC^T, and likewise for B.  Every product is one
call of the library's fused GEMM with trans flags chosen so that no operand is copied or
transposed in memory: the transposes are absorbed by the BLAS op() arguments, i.e. by the
strided loads (and the fused packing) of the kernel itself.

Inputs and outputs are 2-D column-major CUDA tensors (stride(0) == 1), float64 or float32,
as for :func:`paper_2302_08417_gb300.gemm`.
"""
from __future__ import annotations

import torch

from . import gemmfip

_FLIP = {"N": "T", "T": "N"}


def _colmajor(X: torch.Tensor) -> torch.Tensor:
    """X itself if it is a column-major view, else a column-major copy."""
    if X.dim() == 2 and (X.shape[0] <= 1 or X.stride(0) == 1):
        return X
    return X.t().contiguous().t()


def _gemm(A, B, ta, tb, alpha, variant):
    return gemmfip.gemm(_colmajor(A), _colmajor(B), None, alpha, 0.0, ta, tb, variant)


class GemmFunction(torch.autograd.Function):
    """``C = alpha * op(A) * op(B)``; see the module docstring for the backward products."""

    @staticmethod
    def forward(ctx, A, B, transa="N", transb="N", alpha=1.0, variant="fused"):
        ta, tb = transa.upper(), transb.upper()
        ta = "T" if ta == "C" else ta
        tb = "T" if tb == "C" else tb
        ctx.save_for_backward(A, B)
        ctx.conf = (ta, tb, float(alpha), variant)
        return _gemm(A, B, ta, tb, alpha, variant)

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        ta, tb, alpha, variant = ctx.conf
        dC = _colmajor(dC)
        dA = dB = None
        if ctx.needs_input_grad[0]:
            if ta == "N":   # dA = alpha * dC * op(B)^T
                dA = _gemm(dC, B, "N", _FLIP[tb], alpha, variant)
            else:           # dA = alpha * op(B) * dC^T
                dA = _gemm(B, dC, tb, "T", alpha, variant)
        if ctx.needs_input_grad[1]:
            if tb == "N":   # dB = alpha * op(A)^T * dC
                dB = _gemm(A, dC, _FLIP[ta], "N", alpha, variant)
            else:           # dB = alpha * dC^T * op(A)
                dB = _gemm(dC, A, "T", ta, alpha, variant)
        return dA, dB, None, None, None, None


def gemm(A, B, transa="N", transb="N", alpha=1.0, variant="fused"):
    """Differentiable ``alpha * op(A) * op(B)`` on column-major CUDA tensors."""
    return GemmFunction.apply(A, B, transa, transb, alpha, variant)
