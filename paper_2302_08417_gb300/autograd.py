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


def _outputs(shapes, like):
    """Column-major rows x cols tensors for every (rows, cols) in shapes, carved out of one
    allocation (one allocator call per pass instead of one per problem)."""
    total = sum(r * c for r, c in shapes)
    buf = torch.empty(max(total, 1), dtype=like.dtype, device=like.device)
    outs, off = [], 0
    for r, c in shapes:
        outs.append(buf.as_strided((r, c), (1, max(r, 1)), off))
        off += r * c
    return outs


def grad_a_batch(A, B, dC, ta, tb):
    """Arguments of the grouped launch that computes every d op(A_g) (stored shape):
    ta 'N': dA = alpha dC op(B)^T;  ta 'T': dA = alpha op(B) dC^T."""
    xa, xb, ops_a, ops_b = [], [], [], []
    for b, g, x, y in zip(B, dC, ta, tb):
        if x == "N":
            xa.append(g), xb.append(b), ops_a.append("N"), ops_b.append(_FLIP[y])
        else:
            xa.append(b), xb.append(g), ops_a.append(y), ops_b.append("T")
    return ops_a, ops_b, xa, xb, _outputs([tuple(a.shape) for a in A], A[0])


def grad_b_batch(A, B, dC, ta, tb):
    """Arguments of the grouped launch that computes every d op(B_g) (stored shape):
    tb 'N': dB = alpha op(A)^T dC;  tb 'T': dB = alpha dC^T op(A)."""
    xa, xb, ops_a, ops_b = [], [], [], []
    for a, g, x, y in zip(A, dC, ta, tb):
        if y == "N":
            xa.append(a), xb.append(g), ops_a.append(_FLIP[x]), ops_b.append("N")
        else:
            xa.append(g), xb.append(a), ops_a.append("T"), ops_b.append(x)
    return ops_a, ops_b, xa, xb, _outputs([tuple(b.shape) for b in B], B[0])


def forward_batch(A, B, ta, tb):
    """Arguments of the forward grouped launch: C_g = alpha op(A_g) op(B_g)."""
    shapes = [(a.shape[0] if x == "N" else a.shape[1], b.shape[1] if y == "N" else b.shape[0])
              for a, b, x, y in zip(A, B, ta, tb)]
    return ta, tb, A, B, _outputs(shapes, A[0])


class GroupedGemmFunction(torch.autograd.Function):
    """A batch ``C_g = alpha * op(A_g) * op(B_g)`` of uneven problems, each pass one grouped
    launch: the forward products, then in backward all d op(A_g) in one launch and all
    d op(B_g) in another, with the same trans-flag mapping as :class:`GemmFunction`.

    apply(transa, transb, alpha, tile, *A, *B) -> tuple of C_g.  ``tile`` None lets the
    autotuner pick the tile shape of each launch."""

    @staticmethod
    def forward(ctx, transa, transb, alpha, tile, *AB):
        from . import grouped
        count = len(AB) // 2
        A, B = [_colmajor(x) for x in AB[:count]], [_colmajor(x) for x in AB[count:]]
        ta = ["T" if t.upper() == "C" else t.upper() for t in transa]
        tb = ["T" if t.upper() == "C" else t.upper() for t in transb]
        C = []
        if count:
            args = forward_batch(A, B, ta, tb)
            grouped.run_batch(*args, alpha, tile)
            C = args[4]
        ctx.save_for_backward(*A, *B)
        ctx.conf = (ta, tb, float(alpha), tile, count)
        return tuple(C)

    @staticmethod
    def backward(ctx, *dC):
        from . import grouped
        ta, tb, alpha, tile, count = ctx.conf
        saved = ctx.saved_tensors
        A, B = saved[:count], saved[count:]
        dC = [_colmajor(g) for g in dC]
        dA = dB = [None] * count
        if any(ctx.needs_input_grad[4:4 + count]):
            args = grad_a_batch(A, B, dC, ta, tb)
            grouped.run_batch(*args, alpha, tile)
            dA = args[4]
        if any(ctx.needs_input_grad[4 + count:]):
            args = grad_b_batch(A, B, dC, ta, tb)
            grouped.run_batch(*args, alpha, tile)
            dB = args[4]
        return (None, None, None, None, *dA, *dB)


def grouped_gemm(A, B, transa=None, transb=None, alpha=1.0, tile=None):
    """Differentiable batch ``[alpha * op(A_g) * op(B_g)]`` of uneven problems (lists of
    column-major CUDA tensors of one dtype); returns the list of C_g."""
    count = len(A)
    transa = list(transa) if transa is not None else ["N"] * count
    transb = list(transb) if transb is not None else ["N"] * count
    return list(GroupedGemmFunction.apply(transa, transb, alpha, tile, *A, *B))
