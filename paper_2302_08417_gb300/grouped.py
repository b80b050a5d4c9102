"""Grouped GEMM: a batch of independent problems of uneven sizes as one launch.

:class:`Batch` holds the device arrays the C entry points read (problem sizes, operand orders,
leading dimensions, scalars, device pointers, and a processing order, largest problems first).
A :class:`Plan` gives each problem a warp-tile shape and a k-split factor; plans are chosen
per size bucket by :func:`autotune_plan`, which times candidate plans on the batch itself
(coordinate descent over the buckets, on scratch copies of C, whatever beta is) and caches the
choice by the batch's size histogram.  :class:`GraphRunner` captures the call in a CUDA graph
and replays it.  All arithmetic runs in the CUDA library.
"""
from __future__ import annotations

import math
import statistics

import torch

from . import gemmfip as g

_ALL = (g.GFIP_GROUP_TILE_DEFAULT, g.GFIP_GROUP_TILE_SMALL, g.GFIP_GROUP_TILE_TINY,
        g.GFIP_GROUP_TILE_16X8, g.GFIP_GROUP_TILE_8X16)
TILES = {8: _ALL, 4: _ALL}
# warp tile (rows x columns of C) of each tile shape, per element size (as in gfip_grouped.cu)
SHAPES = {(e, t): s for e in (4, 8)
          for t, s in zip(_ALL, ((32, 32), (32, 16), (16, 16), (16, 8), (8, 16)))}
SPLITS = (1, 2, 4)
KC = 8    # k rows per chunk of the warp pipeline (as in gfip_grouped.cu)


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
        self.device = dev
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
        self._args = dict(transa=list(transa), transb=list(transb), alpha=list(alpha),
                          beta=list(beta))
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
        self._orders = {}
        self._keep = (A, B, C)   # the operands must outlive the batch

    def order_for(self, codes) -> torch.Tensor:
        """Processing order for per-problem plan codes: costliest work units first (see
        :func:`unit_cost`), so that the kernel's warps, dealt the units in alternating bands,
        end together."""
        key = tuple(codes)
        if key not in self._orders:
            cost = [unit_cost(self.esz, c & 0xFF, c >> 8, *s) for s, c in zip(self.sizes, codes)]
            rank = sorted(range(self.count), key=lambda q: (-cost[q], q))
            self._orders[key] = torch.tensor(rank, dtype=torch.int32, device=self.device)
        return self._orders[key]

    @property
    def order(self) -> torch.Tensor:
        """The processing order for the default tile shape, unsplit."""
        return self.order_for([g.GFIP_GROUP_PLAN(g.GFIP_GROUP_TILE_DEFAULT, 1)] * self.count)

    def flops(self) -> float:
        return sum(2.0 * m * n * k for m, n, k in self.sizes)

    def with_scratch_c(self) -> "Batch":
        """The same problems writing to fresh copies of C (for timing candidate plans)."""
        A, B, C = self._keep
        Cs = []
        for c in C:
            buf = torch.empty((c.shape[1], c.stride(1)), dtype=c.dtype, device=c.device)
            view = buf.t()[: c.shape[0], :]
            view.copy_(c)
            Cs.append(view)
        return Batch(self._args["transa"], self._args["transb"], A, B, Cs, self._args["alpha"],
                     self._args["beta"])

    def signature(self):
        """Size histogram of the batch: dtype, count and the problem count per size bucket."""
        hist = {}
        for m, n, k in self.sizes:
            b = bucket_of(m, n, k)
            hist[b] = hist.get(b, 0) + 1
        return (self.esz, self.count, tuple(sorted(hist.items())))


def bucket_of(m: int, n: int, k: int):
    """Size bucket of a problem: class of max(m, n) (<= 16, 32, 64, 128, more) and of k
    (< 32, < 128, more)."""
    x = max(m, n)
    sc = 0 if x <= 16 else 1 if x <= 32 else 2 if x <= 64 else 3 if x <= 128 else 4
    kc = 0 if k < 32 else 1 if k < 128 else 2
    return (sc, kc)


def unit_cost(esz: int, tile: int, splits: int, m: int, n: int, k: int) -> int:
    """Relative time of one work unit (one k-range of one warp tile) of a problem: the padded
    multiply-adds of its k chunks, a copy overhead per chunk and an overhead per unit (look-up,
    epilogue).  Only the order of the costs matters."""
    bm, bn = SHAPES[(esz, tile)]
    chunks = math.ceil(math.ceil(max(k, 1) / KC) / max(1, splits))
    return chunks * (bm * bn + 512) + 2 * bm * bn + 2048


class Plan:
    """Warp-tile shape and k-split factor per problem, as the device array the library reads,
    with the processing order that suits it."""

    def __init__(self, batch: Batch, codes):
        self.codes = list(codes)
        self.tensor = torch.tensor(self.codes, dtype=torch.int32, device=batch.device)
        self.order = batch.order_for(self.codes)
        self.split_elems = 0
        for (m, n, k), c in zip(batch.sizes, self.codes):
            tile, splits = c & 0xFF, c >> 8
            bm, bn = SHAPES[(batch.esz, tile)]
            splits = max(1, min(splits, math.ceil(max(k, 1) / KC)))
            if splits > 1 and m > 0 and n > 0:
                self.split_elems += math.ceil(m / bm) * math.ceil(n / bn) * splits * bm * bn

    @classmethod
    def from_buckets(cls, batch: Batch, choice: dict) -> "Plan":
        return cls(batch, [g.GFIP_GROUP_PLAN(*choice[bucket_of(*s)]) for s in batch.sizes])

    @classmethod
    def uniform(cls, batch: Batch, tile: int, splits: int = 1) -> "Plan":
        return cls(batch, [g.GFIP_GROUP_PLAN(tile, splits)] * batch.count)


def _ensure(h, need):
    if h.workspace is None or h.workspace.numel() < need:
        if h.workspace is not None:
            torch.cuda.current_stream().synchronize()
        h._set_ws(need + (1 << 20))


def run(batch: Batch, tile_or_plan, handle: g.Handle | None = None) -> None:
    """Enqueues the grouped GEMM on torch's current stream (asynchronous): every problem with
    one tile shape (an int, GFIP_GROUP_TILE_*), or with the shapes and splits of a Plan."""
    h = handle or g.default_handle()
    h.bind_stream()
    if isinstance(tile_or_plan, Plan):
        plan = tile_or_plan
        _ensure(h, g.gfip_grouped_plan_workspace_size(h.h, batch.count, plan.split_elems,
                                                       batch.esz))
        rc = g.gfip_gemm_grouped_plan(
            batch.esz, h.h, batch.count, batch.transa.data_ptr(), batch.transb.data_ptr(),
            batch.m.data_ptr(), batch.n.data_ptr(), batch.k.data_ptr(), batch.alpha.data_ptr(),
            batch.A.data_ptr(), batch.lda.data_ptr(), batch.B.data_ptr(), batch.ldb.data_ptr(),
            batch.beta.data_ptr(), batch.C.data_ptr(), batch.ldc.data_ptr(),
            plan.tensor.data_ptr(), plan.order.data_ptr(), plan.split_elems)
    else:
        _ensure(h, g.gfip_grouped_workspace_size(h.h, batch.count))
        rc = g.gfip_gemm_grouped(batch.esz, h.h, batch.count, batch.transa.data_ptr(),
                                 batch.transb.data_ptr(), batch.m.data_ptr(), batch.n.data_ptr(),
                                 batch.k.data_ptr(), batch.alpha.data_ptr(), batch.A.data_ptr(),
                                 batch.lda.data_ptr(), batch.B.data_ptr(), batch.ldb.data_ptr(),
                                 batch.beta.data_ptr(), batch.C.data_ptr(),
                                 batch.ldc.data_ptr(), int(tile_or_plan))
    if rc != g.GFIP_OK:
        raise g.GemmError(rc, "gfip_gemm_grouped")


def run_batch(transa, transb, A, B, C, alpha, tile=None, beta=0.0,
              handle: g.Handle | None = None) -> Batch:
    """C_g := alpha op(A_g) op(B_g) + beta C_g for lists of column-major tensors, as one
    grouped launch; ``tile`` None asks :func:`autotune_plan` (which times on scratch copies
    of C, so C is written once).  Returns the batch (it keeps the operands alive)."""
    count = len(A)
    batch = Batch(transa, transb, A, B, C, [alpha] * count, [beta] * count)
    run(batch, autotune_plan(batch, handle) if tile is None else tile, handle)
    return batch


def _time_ms(fn, reps):
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def padded_work(esz: int, tile: int, m: int, n: int, k: int) -> int:
    """Multiply-adds a problem costs in a tile shape, padding of m, n and k included."""
    bm, bn = SHAPES[(esz, tile)]
    return math.ceil(m / bm) * bm * math.ceil(n / bn) * bn * max(k, 1)


def _initial_tiles(batch: Batch) -> dict:
    """Per bucket, the tile shape with the least padded work over the bucket's problems (the
    larger tile on a tie): the start of the search, and what bounds FP64 (DFMA-bound)."""
    work = {}
    for m, n, k in batch.sizes:
        b = bucket_of(m, n, k)
        w = work.setdefault(b, {t: 0 for t in TILES[batch.esz]})
        for t in w:
            w[t] += padded_work(batch.esz, t, m, n, k)
    return {b: min(sorted(w), key=lambda t: w[t]) for b, w in work.items()}


_tuned: dict = {}


def autotune_plan(batch: Batch, handle: g.Handle | None = None, reps: int = 3) -> Plan:
    """Per size bucket, the tile shape and k-split factor that make the whole batch fastest.

    Starts from the fastest of two kinds of plan, unsplit: the tile with the least padded work
    in each bucket, or one tile shape for every problem.  Then visits the buckets in
    order of their share of the flops and, for each, times every candidate (each tile shape;
    with k >= 32 also 2- and 4-way splits) with the other buckets held, keeping the fastest.
    Timings run on scratch copies of C, so the caller's C is untouched whatever beta is.  The
    choice is cached by :meth:`Batch.signature`."""
    key = batch.signature()
    if key in _tuned:
        return Plan.from_buckets(batch, _tuned[key])
    flops = {}
    for m, n, k in batch.sizes:
        b = bucket_of(m, n, k)
        flops[b] = flops.get(b, 0.0) + 2.0 * m * n * k
    start = _initial_tiles(batch)
    scratch = batch.with_scratch_c()
    h = handle or g.default_handle()

    def cost(ch):
        plan = Plan.from_buckets(scratch, ch)
        return _time_ms(lambda: run(scratch, plan, h), reps)

    # start from the fastest of: the least padded tile per bucket, or one tile everywhere
    starts = [{b: (start[b], 1) for b in flops}]
    starts += [{b: (t, 1) for b in flops} for t in TILES[batch.esz]]
    best_ms, choice = min(((cost(ch), i) for i, ch in enumerate(starts)))
    choice = starts[choice]
    for b in sorted(flops, key=lambda b: -flops[b]):
        splits = SPLITS if b[1] >= 1 else (1,)
        for tile in TILES[batch.esz]:
            for s in splits:
                if (tile, s) == choice[b]:
                    continue
                trial = dict(choice)
                trial[b] = (tile, s)
                ms = cost(trial)
                if ms < best_ms:
                    best_ms, choice = ms, trial
    _tuned[key] = choice
    return Plan.from_buckets(batch, choice)


def autotune(batch: Batch, handle: g.Handle | None = None, reps: int = 3):
    """The tuned plan of the batch (see :func:`autotune_plan`)."""
    return autotune_plan(batch, handle, reps)


class GraphRunner:
    """The grouped call of one batch captured in a CUDA graph; replay() re-runs it.

    The captured launches point into the handle's workspace, so the runner owns a handle of
    its own by default (a shared handle must not grow its workspace while the graph lives)."""

    def __init__(self, batch: Batch, tile_or_plan, handle: g.Handle | None = None):
        self.batch = batch
        self.plan = tile_or_plan
        self.handle = handle or g.Handle()
        run(batch, tile_or_plan, self.handle)   # sizes the workspace before capture
        torch.cuda.synchronize()
        self.stream = torch.cuda.Stream()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(self.stream):
            self.handle.bind_stream(self.stream)
            with torch.cuda.graph(self.graph, stream=self.stream):
                run(batch, tile_or_plan, self.handle)
        self.handle.bind_stream(torch.cuda.current_stream())

    def replay(self):
        self.graph.replay()
