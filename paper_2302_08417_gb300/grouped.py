"""Grouped GEMM: a batch of independent problems of uneven sizes as one launch.

:class:`Batch` holds the device arrays the C entry points ``gfip_dgemm_grouped`` /
``gfip_sgemm_grouped`` read (problem sizes, operand orders, leading dimensions, scalars and
device pointers), :func:`autotune` picks the tile shape for a batch by timing every compiled
shape on that batch (results cached by a size signature), and :class:`GraphRunner` captures
the call in a CUDA graph and replays it.  All arithmetic runs in the CUDA library.
"""
from __future__ import annotations

import math

import torch

from . import gemmfip as g

TILES = {8: (g.GFIP_GROUP_TILE_DEFAULT,),
         4: (g.GFIP_GROUP_TILE_DEFAULT, g.GFIP_GROUP_TILE_SMALL)}


class Batch:
    """Device-side description of ``count`` problems C_g := alpha_g op(A_g) op(B_g) + beta_g C_g.

    ``A``, ``B``, ``C`` are sequences of column-major 2-D CUDA tensors (stride(0) == 1) in the
    stored shapes (A is m x k for 'N', k x m for 'T'); the other arguments are sequences of
    per-problem values."""

    def __init__(self, transa, transb, A, B, C, alpha, beta):
        count = len(A)
        if not (len(B) == len(C) == len(transa) == len(transb) == len(alpha) == len(beta)
                == count):
            raise ValueError("all per-problem sequences must have the same length")
        dtype = A[0].dtype if count else torch.float64
        dev = A[0].device if count else torch.device("cuda")
        self.count = count
        self.dtype = dtype
        self.esz = 8 if dtype == torch.float64 else 4
        ms, ns, ks = [], [], []
        for ta, tb, a, b in zip(transa, transb, A, B):
            m = a.shape[0] if ta in "Nn" else a.shape[1]
            kk = a.shape[1] if ta in "Nn" else a.shape[0]
            n = b.shape[1] if tb in "Nn" else b.shape[0]
            ms.append(m)
            ns.append(n)
            ks.append(kk)
        self.sizes = list(zip(ms, ns, ks))

        def ld(x):
            if x.dim() == 2 and x.stride(0) == 1 and x.stride(1) >= max(1, x.shape[0]):
                return x.stride(1)
            return g._colmajor_ld(x, "matrix")

        i32 = dict(dtype=torch.int32, device=dev)
        i64 = dict(dtype=torch.int64, device=dev)
        self.transa = torch.tensor([ord(t) for t in transa], dtype=torch.uint8, device=dev)
        self.transb = torch.tensor([ord(t) for t in transb], dtype=torch.uint8, device=dev)
        self.m = torch.tensor(ms, **i32)
        self.n = torch.tensor(ns, **i32)
        self.k = torch.tensor(ks, **i32)
        self.alpha = torch.tensor(list(alpha), dtype=dtype, device=dev)
        self.beta = torch.tensor(list(beta), dtype=dtype, device=dev)
        self.A = torch.tensor([x.data_ptr() for x in A], **i64)
        self.B = torch.tensor([x.data_ptr() for x in B], **i64)
        self.C = torch.tensor([x.data_ptr() for x in C], **i64)
        self.lda = torch.tensor([ld(x) for x in A], **i64)
        self.ldb = torch.tensor([ld(x) for x in B], **i64)
        self.ldc = torch.tensor([ld(x) for x in C], **i64)
        self._keep = (A, B, C)   # the operands must outlive the batch

    def flops(self) -> float:
        return sum(2.0 * m * n * k for m, n, k in self.sizes)

    def signature(self):
        """Size bucket of the batch: dtype, count, log2 buckets of the median m, n, k."""
        def med(i):
            v = sorted(s[i] for s in self.sizes)
            return int(math.log2(max(1, v[len(v) // 2]))) if v else 0
        return (self.esz, self.count, med(0), med(1), med(2))


def run(batch: Batch, tile: int, handle: g.Handle | None = None) -> None:
    """Enqueues the grouped GEMM on torch's current stream (asynchronous)."""
    h = handle or g.default_handle()
    h.bind_stream()
    need = g.gfip_grouped_workspace_size(h.h, batch.count)
    if h.workspace is None or h.workspace.numel() < need:
        if h.workspace is not None:
            torch.cuda.current_stream().synchronize()
        h._set_ws(need + (1 << 20))
    rc = g.gfip_gemm_grouped(batch.esz, h.h, batch.count, batch.transa.data_ptr(),
                             batch.transb.data_ptr(), batch.m.data_ptr(), batch.n.data_ptr(),
                             batch.k.data_ptr(), batch.alpha.data_ptr(), batch.A.data_ptr(),
                             batch.lda.data_ptr(), batch.B.data_ptr(), batch.ldb.data_ptr(),
                             batch.beta.data_ptr(), batch.C.data_ptr(), batch.ldc.data_ptr(),
                             tile)
    if rc != g.GFIP_OK:
        raise g.GemmError(rc, "gfip_gemm_grouped")


def run_batch(transa, transb, A, B, C, alpha, tile=None, beta=0.0,
              handle: g.Handle | None = None) -> Batch:
    """C_g := alpha op(A_g) op(B_g) + beta C_g for lists of column-major tensors, as one
    grouped launch; ``tile`` None asks :func:`autotune` (which, with beta == 0, may overwrite
    C while timing).  Returns the batch (it keeps the operands alive)."""
    count = len(A)
    batch = Batch(transa, transb, A, B, C, [alpha] * count, [beta] * count)
    if tile is None:
        tile = autotune(batch, handle) if beta == 0.0 else TILES[batch.esz][0]
    run(batch, tile, handle)
    return batch


_tuned: dict = {}


def autotune(batch: Batch, handle: g.Handle | None = None, reps: int = 3) -> int:
    """Times every compiled tile shape on this batch and returns the fastest; the choice is
    cached per :meth:`Batch.signature`.  The timed runs overwrite C (beta is applied each
    time), so tune on scratch output buffers or restore C afterwards."""
    key = batch.signature()
    if key in _tuned:
        return _tuned[key]
    best, best_ms = None, float("inf")
    for tile in TILES[batch.esz]:
        run(batch, tile, handle)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            run(batch, tile, handle)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        if ms < best_ms:
            best, best_ms = tile, ms
    _tuned[key] = best
    return best


class GraphRunner:
    """The grouped call of one batch captured in a CUDA graph; replay() re-runs it.

    The captured launches point into the handle's workspace, so the runner owns a handle of
    its own by default (a shared handle must not grow its workspace while the graph lives)."""

    def __init__(self, batch: Batch, tile: int, handle: g.Handle | None = None):
        self.batch = batch
        self.handle = handle or g.Handle()
        run(batch, tile, self.handle)          # sizes the workspace before capture
        torch.cuda.synchronize()
        self.stream = torch.cuda.Stream()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(self.stream):
            self.handle.bind_stream(self.stream)
            with torch.cuda.graph(self.graph, stream=self.stream):
                run(batch, tile, self.handle)
        self.handle.bind_stream(torch.cuda.current_stream())

    def replay(self):
        self.graph.replay()
