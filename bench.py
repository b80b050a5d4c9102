"""Benchmark of the fused-in-packing GEMM on GB300.

One step = one C := alpha*op(A)*op(B) + beta*C call of the fused FP64 routine on the
headline workload (m = n = k = 8192, transa = transb = 'N', lda = ldb = ldc = 8199 -- not
16-byte aligned -- alpha = 1, beta = 0.5, entries uniform[-1, 1]).  The three operands
(1.6 GB) are larger than the 129 MB L2, so no flush is needed between steps.

Prints ONE JSON line: GFLOP/s over the timed steps (device time, CUDA events), the roofline
of the dominant kernel against the FP64 DFMA rate, the end-to-end figure through the public
API with host buffers, the oracle timed on the host cores on a bounded sample, the SM clocks
seen during the timed region, the fused-vs-plain spectrum over all 20 sizes in both dtypes
(with per-size noise bands), and, last, a compact summary of all of it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-spectrum]

With N > 1 (launched by torchrun) every rank runs an independent replica of the workload
(GEMM is not sharded here); the value is the total over ranks divided by the slowest rank.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M = N = K = 8192     # headline size; --size overrides it (profiling of smaller cases)
PAD = 7
ALPHA, BETA = 1.0, 0.5
SMS = 152
DFMA_FLOP_PER_CLK_PER_SM = 4      # 2 DFMA lanes per clock per SM (measured by peak_probe)
FFMA_FLOP_PER_CLK_PER_SM = 256    # 128 FFMA lanes per clock per SM
SM_MAX_MHZ = 2070.0
FP64_PEAK_GFLOPS = SMS * DFMA_FLOP_PER_CLK_PER_SM * SM_MAX_MHZ / 1e3   # 1258.6
FP32_PEAK_GFLOPS = SMS * FFMA_FLOP_PER_CLK_PER_SM * SM_MAX_MHZ / 1e3   # 80547.8
HBM_GBS = 6785.2
def workload(dtype="f64", size=8192, variant="fused") -> str:
    return (f"{dtype} gemm m=n=k={size} N/N lda=ldb=ldc={size + PAD} alpha=1 beta=0.5 "
            f"uniform[-1,1] {variant}")


WORKLOAD = workload()

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the FP64 GEMM
# kernel on this workload, from a one-pass ncu capture of the full-size launch (summary in
# profiles/); valid only while the kernel sources hash to kernel_hash.
TRAFFIC = {"bytes_per_launch": 23.14e9 + 1.65e9, "kernel_hash": "26b705248ccb94c3"}
KERNEL_SOURCES = ["paper_2302_08417_gb300/csrc/gfip_kernels.cuh",
                  "paper_2302_08417_gb300/csrc/gfip_internal.h"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def gflop(m=None, n=None, k=None) -> float:
    m, n, k = (M if m is None else m), (N if n is None else n), (K if k is None else k)
    return 2.0 * m * n * k / 1e9


def algorithmic_bytes(s=8, beta=BETA) -> int:
    """Read A, read B, read C (beta != 0), write C: the bytes the GEMM must move."""
    return s * (M * K + K * N + M * N * (1 + (beta != 0.0)))


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v: float) -> float:
    """The largest v over the ranks (the slowest rank's time); a CUDA tensor on NCCL, a host
    tensor on other backends."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_operands(seed: int, dtype, m=None, n=None, k=None, pad=PAD):
    """Column-major operands on the GPU, uniform[-1, 1], leading dimension rows + pad."""
    import torch
    m, n, k = (M if m is None else m), (N if n is None else n), (K if k is None else k)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    ld_a, ld_b, ld_c = m + pad, k + pad, m + pad

    def mat(rows, cols, ld):
        buf = torch.rand((cols, ld), generator=g, dtype=dtype, device="cuda") * 2 - 1
        return buf.t()[:rows, :]   # rows x cols view, stride (1, ld), over a (cols, ld) buffer
    return mat(m, k, ld_a), mat(k, n, ld_b), mat(m, n, ld_c)


def host_copy(X):
    """Pinned host copy of a column-major view with the same leading dimension."""
    import torch
    rows, cols = X.shape
    ld = X.stride(1)
    buf = torch.empty((cols, ld), dtype=X.dtype, pin_memory=True)
    buf.t()[:rows, :].copy_(X)
    return buf.t()[:rows, :], buf


def cpu_oracle_sample(A_host, B_host, C_host, m, k, lda, ldb, ldc, budget_s=12.0):
    """Times the oracle on the host cores on the first columns of the same workload."""
    import numpy as np
    import oracle
    threads = os.cpu_count() or 1
    oracle.build()

    def run(cols):
        Bs = np.ascontiguousarray(B_host[: ldb * cols])
        Cs = np.ascontiguousarray(C_host[: ldc * cols])
        t0 = time.perf_counter()
        rc = oracle.gemm("N", "N", m, cols, k, ALPHA, A_host, lda, Bs, ldb, BETA, Cs, ldc,
                         nthreads=threads)
        dt = time.perf_counter() - t0
        assert rc == 0
        return dt

    cols = threads
    dt = run(cols)
    while dt < 1.0 and cols * 4 <= N:
        cols *= 4
        dt = run(cols)
    target = int(min(N, max(cols, cols * budget_s / max(dt, 1e-6))))
    target = max(threads, target // threads * threads)
    dt = run(target)
    return {"value": round(gflop(m, target, k) / dt, 3), "unit": "GFLOP/s", "cores": threads,
            "kind": "oracle",
            "sample": f"first {target} of {N} columns of C (m=k={m}, same operands), "
                      f"{dt:.1f} s, FP64 j-p-i triple loop, OpenMP over columns"}


def oracle_single_thread(sizes=(256, 512, 1024, 2048)):
    """The oracle on ONE host core (the paper's single-core framing) for m = n = k <= 2048,
    N/N, ld = m + 7, alpha 1, beta 0.5, uniform[-1, 1]; the headline size is extrapolated
    from the largest one as n^3 and labelled so."""
    import numpy as np
    import oracle
    from paper_2302_08417_gb300 import inputs
    oracle.build()
    out = {"note": "one thread, FP64 j-p-i triple loop; seconds per call and GFLOP/s"}
    last = None
    for n in sizes:
        p = inputs.problem(n, "N", "N", n, n, n, ALPHA, BETA, PAD, PAD, PAD)
        C = p.C0.copy()
        t0 = time.perf_counter()
        rc = oracle.gemm("N", "N", n, n, n, ALPHA, p.A, p.lda, p.B, p.ldb, BETA, C, p.ldc,
                         nthreads=1)
        dt = time.perf_counter() - t0
        assert rc == 0
        out[str(n)] = {"s": round(dt, 4), "gflops": round(gflop(n, n, n) / dt, 3)}
        last = (n, dt)
    n0, t0_ = last
    out["8192_extrapolated_s"] = round(t0_ * (8192 / n0) ** 3, 1)
    out["8192_extrapolated_note"] = f"extrapolated as n^3 from {n0}, not measured"
    return out


VARIANTS = ("fused", "direct", "pack_then_compute")


class VariantTimer:
    """Device time per call of one GEMM call shape in each variant.  Calls shorter than half a
    millisecond are captured R at a time (R calls >= target_ms) in one CUDA graph per variant
    and replayed; longer ones are timed as single calls.  Each timing is one replay (or call)
    between two CUDA events on the launching stream."""

    def __init__(self, h, g, torch, esz, ta, tb, m, n, k, A, lda, B, ldb, beta, C, ldc,
                 target_ms=2.0):
        import math
        self.torch, self.h = torch, h
        self.fns, self.reps = {}, {}
        for var in VARIANTS:
            name = g.ENTRY[(var, esz)]

            def call(name=name):
                rc = g._gemm_call(name, h.h, ta, tb, m, n, k, ALPHA, A.data_ptr(), lda,
                                  B.data_ptr(), ldb, beta, C.data_ptr(), ldc)
                if rc != 0:
                    raise g.GemmError(rc, name)
            one = self._events_ms(call)     # the first call also warms up
            if one > 0.5:
                self.fns[var], self.reps[var] = call, 1
                continue
            R = max(1, min(400, math.ceil(target_ms / max(one, 1e-3))))

            def burst(call=call, R=R):
                for _ in range(R):
                    call()
            stream = torch.cuda.Stream()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.stream(stream):
                h.bind_stream(stream)
                with torch.cuda.graph(graph, stream=stream):
                    burst()
            h.bind_stream()
            graph.replay()
            torch.cuda.synchronize()
            self.fns[var], self.reps[var] = graph.replay, R
            setattr(self, f"_graph_{var}", graph)

    def _events_ms(self, fn):
        torch = self.torch
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1)

    def run(self, rounds):
        """Per variant: the device times per call of `rounds` timings, taken round-robin over
        the variants so that clock or thermal drift touches all of them alike."""
        out = {v: [] for v in VARIANTS}
        for _ in range(rounds):
            for v in VARIANTS:
                out[v].append(self._events_ms(self.fns[v]) / self.reps[v])
        return out


def summarize(times, gflop_per_call, peak):
    """Median GFLOP/s per variant, fused / best plain variant, and the noise band: the largest
    relative spread (max - min) / median of the timings of any variant."""
    med = {v: statistics.median(t) for v, t in times.items()}
    gf = {v: gflop_per_call / (med[v] * 1e-3) for v in med}
    noise = max((max(t) - min(t)) / statistics.median(t) for t in times.values())
    best_plain = max(gf["direct"], gf["pack_then_compute"])
    return {"gflops": {v: round(gf[v], 2) for v in VARIANTS},
            "dev_us": {v: round(med[v] * 1e3, 2) for v in VARIANTS},
            "fused_over_best_plain": round(gf["fused"] / best_plain, 4),
            "noise": round(noise, 4), "frac": round(gf["fused"] / peak, 4)}


def sweep(h, g, torch, sizes, dtypes=("f64", "f32"), rounds=7, long_rounds=3):
    """The fused-vs-plain size spectrum, N/N, ld = m + 7, alpha 1, beta 0.5, uniform[-1, 1]:
    every size of the 16..16384 spectrum in FP64 and FP32, the three variants timed
    round-robin (`rounds` rounds, `long_rounds` when one call takes over 100 ms).  Operands of
    the sizes below about 2048 stay in L2 between calls (warm), as they would in a loop of
    calls."""
    out = {"note": "N/N, ld = m + 7, alpha 1, beta 0.5, uniform[-1,1]; median device time "
                   "per call over rounds of graph-replayed calls; noise = largest (max-min)/"
                   "median of a variant's timings"}
    for tag in dtypes:
        dtype = torch.float64 if tag == "f64" else torch.float32
        esz = 8 if tag == "f64" else 4
        peak = FP64_PEAK_GFLOPS if tag == "f64" else FP32_PEAK_GFLOPS
        rows = {}
        for n in sizes:
            A, B, C = make_operands(n, dtype, n, n, n)
            ld = n + PAD
            h.ensure_workspace("N", "N", n, n, n, esz)
            vt = VariantTimer(h, g, torch, esz, "N", "N", n, n, n, A, ld, B, ld, BETA, C, ld)
            at_peak_s = 2.0 * n * n * n / (peak * 1e9)
            r = rounds if at_peak_s < 0.1 else (long_rounds if at_peak_s < 1.0 else 2)
            rows[str(n)] = summarize(vt.run(r), gflop(n, n, n), peak)
            del vt, A, B, C
            torch.cuda.empty_cache()
        out[tag] = rows
    out["status"] = h.status()
    return out


# Configurations beside the square N/N spectrum: the 256^3 workload with every leading
# dimension exactly 256 (C1), transposed operand orders, beta = 0, unpadded ld.
EXTRA_CASES = [
    # (tag, dtype, transa, transb, m, n, k, pad, beta)
    ("C1 f64 N/N 256 ld=256 beta=0.5", "f64", "N", "N", 256, 256, 256, 0, 0.5),
    ("f64 T/T 2048 ld=m+7 beta=0", "f64", "T", "T", 2048, 2048, 2048, 7, 0.0),
    ("f64 N/T 8192x8192x64 ld=m beta=0.5", "f64", "N", "T", 8192, 8192, 64, 0, 0.5),
    ("f32 T/N 4096 ld=m beta=0", "f32", "T", "N", 4096, 4096, 4096, 0, 0.0),
    ("f32 N/T 1536 ld=m+7 beta=0.5", "f32", "N", "T", 1536, 1536, 1536, 7, 0.5),
    ("f32 T/N 64x8192x8192 ld=m+7 beta=0", "f32", "T", "N", 64, 8192, 8192, 7, 0.0),
]


def extra_cases(h, g, torch, rounds=7):
    out = {}
    for tag, dt, ta, tb, m, n, k, pad, beta in EXTRA_CASES:
        dtype = torch.float64 if dt == "f64" else torch.float32
        esz = 8 if dt == "f64" else 4
        peak = FP64_PEAK_GFLOPS if dt == "f64" else FP32_PEAK_GFLOPS
        gen = torch.Generator(device="cuda")
        gen.manual_seed(m + n + k)

        def mat(rows, cols):
            ld = rows + pad
            buf = torch.rand((cols, ld), generator=gen, dtype=dtype, device="cuda") * 2 - 1
            return buf.t()[:rows, :]
        A = mat(m, k) if ta == "N" else mat(k, m)
        B = mat(k, n) if tb == "N" else mat(n, k)
        C = mat(m, n)
        h.ensure_workspace(ta, tb, m, n, k, esz)
        vt = VariantTimer(h, g, torch, esz, ta, tb, m, n, k, A, A.stride(1), B, B.stride(1),
                          beta, C, C.stride(1))
        out[tag] = summarize(vt.run(rounds), gflop(m, n, k), peak)
        del vt, A, B, C
    return out


def sweep_markdown(res) -> str:
    lines = []
    for tag in ("f64", "f32"):
        if tag not in res:
            continue
        lines.append(f"| {tag} n | fused GF/s | direct GF/s | pack-then-compute GF/s | "
                     "fused / best plain | noise | fused frac of peak | fused us |")
        lines.append("|---|---|---|---|---|---|---|---|")
        for n, r in res[tag].items():
            gf = r["gflops"]
            lines.append(f"| {n} | {gf['fused']} | {gf['direct']} | {gf['pack_then_compute']} "
                         f"| {r['fused_over_best_plain']} | {r['noise']} | {r['frac']} | "
                         f"{r['dev_us']['fused']} |")
        lines.append("")
    return "\n".join(lines)


def emulation_report(h, g, torch, n=8192, slice_counts=(3, 5, 7, 9), samples=2048):
    """FP64 emulated on the tensor cores (gfip_dgemm_ozaki): GFLOP/s (FP64-equivalent, 2n^3 per
    call, device time) and the error against the oracle on sampled entries, for uniform[-1,1]
    and log-uniform [1e-4, 1e4] magnitudes with random sign."""
    import numpy as np
    import oracle
    ld = n + PAD
    out = {"n": n, "note": "N/N, ld = n + 7, alpha 1, beta 0.5; error = max over sampled "
           "entries of |C - C_oracle| / (|alpha||A||B| + |beta||C0|) entrywise"}
    gen = torch.Generator(device="cuda")
    gen.manual_seed(99)
    for dist in ("uniform", "logmag"):
        def mat():
            u = torch.rand((n, ld), generator=gen, dtype=torch.float64, device="cuda")
            if dist == "uniform":
                return u * 2 - 1
            mag = torch.pow(10.0, torch.rand((n, ld), generator=gen, dtype=torch.float64,
                                             device="cuda") * 8 - 4)
            return torch.where(u < 0.5, -mag, mag)
        A, B, C0 = mat(), mat(), mat()
        hA = A.cpu().numpy().reshape(-1)
        hB = B.cpu().numpy().reshape(-1)
        hC0 = C0.cpu().numpy().reshape(-1)
        rng = np.random.Generator(np.random.PCG64(5))
        ii = rng.integers(0, n, samples)
        jj = rng.integers(0, n, samples)
        threads = os.cpu_count() or 1
        ref = oracle.entries("N", "N", n, n, n, 1.0, hA, ld, hB, ld, BETA, hC0, ld, ii, jj,
                             nthreads=threads)
        mag = oracle.entries("N", "N", n, n, n, 1.0, hA, ld, hB, ld, BETA, hC0, ld, ii, jj,
                             absval=True, nthreads=threads)
        rows = {}
        for S in slice_counts:
            h.ensure_ozaki_workspace(n, n, n, S)
            C = C0.clone()

            def call():
                rc = g.gfip_dgemm_ozaki(h.h, "N", "N", n, n, n, 1.0, A.data_ptr(), ld,
                                        B.data_ptr(), ld, BETA, C.data_ptr(), ld, S)
                assert rc == 0, rc
            C.copy_(C0)
            call()
            torch.cuda.synchronize()
            got = C.cpu().numpy().reshape(-1)[ii + jj * ld]
            err = np.abs(got - ref) / mag
            best = float("inf")
            for _ in range(2):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                call()
                e1.record()
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
            gf = gflop(n, n, n) / (best * 1e-3)
            rows[f"slices_{S}"] = {"gflops": round(gf, 1),
                                   "speedup_vs_dfma_peak": round(gf / FP64_PEAK_GFLOPS, 2),
                                   "max_rel_err": float(f"{err.max():.3e}"),
                                   "median_rel_err": float(f"{np.median(err):.3e}")}
        out[dist] = rows
        del A, B, C0
    out["status"] = h.status()
    return out


def batched_report(g, torch, count=4096, seed=11):
    """Grouped GEMM on the batched workload: `count` problems, m, n, k log-uniform in
    [4, 256], random operand orders, leading dimensions rows + {0..7}, FP64 and FP32.
    Reports GFLOP/s of one grouped launch replayed from a CUDA graph (tile chosen by the
    autotuner), against the same problems as `count` single-GEMM calls (direct variant)
    captured in one CUDA graph and issued eagerly from Python."""
    import numpy as np
    from paper_2302_08417_gb300 import grouped as gr
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.exp(rng.uniform(np.log(4), np.log(256), (count, 3))).round().astype(int)
    ta = rng.choice(["N", "T"], count)
    tb = rng.choice(["N", "T"], count)
    pads = rng.integers(0, 8, (count, 3))
    out = {"problems": count, "note": "m, n, k log-uniform in [4, 256], random trans, "
           "ld = rows + {0..7}, alpha 1, beta 0.5; CUDA events around graph replays"}
    for dtype, tag in ((torch.float64, "f64"), (torch.float32, "f32")):
        gen = torch.Generator(device="cuda")
        gen.manual_seed(seed)
        A, B, C = [], [], []
        for q in range(count):
            m, n, k = (int(x) for x in sizes[q])
            ra, ca = (m, k) if ta[q] == "N" else (k, m)
            rb, cb = (k, n) if tb[q] == "N" else (n, k)

            def mk(rows, cols, pad):
                ld = rows + int(pad)
                buf = torch.rand((cols, ld), generator=gen, dtype=dtype, device="cuda")
                return buf.t()[:rows, :]
            A.append(mk(ra, ca, pads[q, 0]))
            B.append(mk(rb, cb, pads[q, 1]))
            C.append(mk(m, n, pads[q, 2]))
        batch = gr.Batch(list(ta), list(tb), A, B, C, [1.0] * count, [BETA] * count)
        flops = batch.flops()
        t0 = time.perf_counter()
        plan = gr.autotune_plan(batch)
        tune_s = time.perf_counter() - t0
        runner = gr.GraphRunner(batch, plan)

        def timed(fn, reps=5):
            fn()
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
            return best
        grouped_ms = timed(runner.replay)
        # baseline: one single-GEMM launch per problem, captured in a CUDA graph
        h = g.Handle()
        esz = 8 if dtype == torch.float64 else 4
        entry = g.ENTRY[("direct", esz)]
        maxw = max(g.gfip_workspace_size(h.h, ta[q], tb[q], *(int(x) for x in sizes[q]), esz)
                   for q in range(count))
        h._set_ws(maxw + (1 << 20))

        def singles():
            for q in range(count):
                m, n, k = (int(x) for x in sizes[q])
                rc = g._gemm_call(entry, h.h, ta[q], tb[q], m, n, k, 1.0, A[q].data_ptr(),
                                  A[q].stride(1), B[q].data_ptr(), B[q].stride(1), BETA,
                                  C[q].data_ptr(), C[q].stride(1))
                assert rc == 0, rc
        h.bind_stream()
        singles()
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            h.bind_stream(s)
            with torch.cuda.graph(graph, stream=s):
                singles()
        h.bind_stream()
        singles_graph_ms = timed(graph.replay)
        singles_eager_ms = timed(singles, reps=2)
        choice = gr._tuned.get(batch.signature(), {})
        peak = FP64_PEAK_GFLOPS if tag == "f64" else FP32_PEAK_GFLOPS
        gf_grouped = flops / 1e9 / (grouped_ms * 1e-3)
        out[tag] = {"plan": {f"{b[0]}/{b[1]}": list(v) for b, v in sorted(choice.items())},
                    "plan_note": "size bucket (max(m,n) class <=16,32,64,128,more / k class "
                                 "<32,<128,more) -> [tile shape, k-splits]",
                    "tune_s": round(tune_s, 2), "gflop_per_batch": round(flops / 1e9, 3),
                    "grouped_graph_gflops": round(gf_grouped, 1),
                    "frac_of_peak": round(gf_grouped / peak, 4),
                    "singles_graph_gflops": round(flops / 1e9 / (singles_graph_ms * 1e-3), 1),
                    "singles_eager_gflops": round(flops / 1e9 / (singles_eager_ms * 1e-3), 1),
                    "grouped_ms": round(grouped_ms, 3),
                    "speedup_vs_singles_graph": round(singles_graph_ms / grouped_ms, 2)}
        del runner, graph, A, B, C, batch
    return out


def autograd_report(torch, shapes=((4096, 4096, 1024), (1024, 8192, 4096)), count=1024,
                    seed=13):
    """Differentiable GEMM, forward + backward (three products, 6mnk flop) per step: the
    fused kernel through autograd.gemm, the direct variant, and torch.matmul (cuBLAS, TF32
    off) for context, at the two single shapes (N/N); then a batch of `count` uneven problems
    (m, n, k log-uniform in [8, 128], random trans) as three grouped launches
    (autograd.grouped_gemm) against one autograd.gemm call per problem.  Device time, CUDA
    events, best of 3 after a warm-up."""
    import numpy as np
    from paper_2302_08417_gb300 import autograd as ag
    torch.backends.cuda.matmul.allow_tf32 = False

    def best_ms(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    out = {"note": "forward + backward = 3 GEMMs (6mnk flop); device time, best of 3"}
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    for dtype, tag in ((torch.float64, "f64"), (torch.float32, "f32")):
        rows = {}
        for m, n, k in shapes:
            At = (torch.rand((k, m), generator=gen, dtype=dtype, device="cuda") * 2 - 1)
            Bt = (torch.rand((n, k), generator=gen, dtype=dtype, device="cuda") * 2 - 1)
            At.requires_grad_()
            Bt.requires_grad_()
            dC = torch.rand((n, m), generator=gen, dtype=dtype, device="cuda").t() * 2 - 1
            flop = 6.0 * m * n * k

            def step(kind):
                def run():
                    At.grad = None
                    Bt.grad = None
                    if kind == "cublas":
                        C = At.t() @ Bt.t()
                    else:
                        C = ag.gemm(At.t(), Bt.t(), "N", "N", 1.0, kind)
                    C.backward(dC)
                return run
            r = {kind: round(flop / 1e9 / (best_ms(step(kind)) * 1e-3), 1)
                 for kind in ("fused", "direct", "cublas")}
            r["fused_over_cublas"] = round(r["fused"] / r["cublas"], 3)
            rows[f"{m}x{n}x{k}"] = r
            del At, Bt, dC
        # the uneven batch
        rng = np.random.Generator(np.random.PCG64(seed))
        sizes = np.exp(rng.uniform(np.log(8), np.log(128), (count, 3))).round().astype(int)
        ta = [str(x) for x in rng.choice(["N", "T"], count)]
        tb = [str(x) for x in rng.choice(["N", "T"], count)]
        As, Bs = [], []
        for q in range(count):
            m, n, k = (int(x) for x in sizes[q])
            ra, ca = (m, k) if ta[q] == "N" else (k, m)
            rb, cb = (k, n) if tb[q] == "N" else (n, k)
            As.append(torch.rand((ca, ra), generator=gen, dtype=dtype, device="cuda")
                      .requires_grad_())
            Bs.append(torch.rand((cb, rb), generator=gen, dtype=dtype, device="cuda")
                      .requires_grad_())
        dCs = [torch.rand((int(s[1]), int(s[0])), generator=gen, dtype=dtype,
                          device="cuda").t() for s in sizes]
        flop = float(sum(6.0 * int(s[0]) * int(s[1]) * int(s[2]) for s in sizes))

        def grouped_step():
            Cs = ag.grouped_gemm([a.t() for a in As], [b.t() for b in Bs], ta, tb, 1.0)
            torch.autograd.backward(Cs, dCs)

        def singles_step():
            Cs = [ag.gemm(a.t(), b.t(), x, y, 1.0) for a, b, x, y in zip(As, Bs, ta, tb)]
            torch.autograd.backward(Cs, dCs)
        grouped_step()   # tunes the tiles once
        g_ms = best_ms(grouped_step)
        s_ms = best_ms(singles_step, reps=2)
        # device time of the three grouped passes alone: each launch captured in a CUDA graph
        from paper_2302_08417_gb300 import grouped as gr
        At_ = [a.detach().t() for a in As]
        Bt_ = [b.detach().t() for b in Bs]
        passes = [ag.forward_batch(At_, Bt_, ta, tb), ag.grad_a_batch(At_, Bt_, dCs, ta, tb),
                  ag.grad_b_batch(At_, Bt_, dCs, ta, tb)]
        runners = []
        for ops_a, ops_b, xa, xb, outs in passes:
            batch = gr.Batch(ops_a, ops_b, xa, xb, outs, [1.0] * count, [0.0] * count)
            runners.append(gr.GraphRunner(batch, gr.autotune(batch)))
        d_ms = best_ms(lambda: [r.replay() for r in runners])
        rows[f"batch{count}"] = {
            "step_gflops": round(flop / 1e9 / (g_ms * 1e-3), 1),
            "singles_step_gflops": round(flop / 1e9 / (s_ms * 1e-3), 1),
            "step_ms": round(g_ms, 3), "singles_step_ms": round(s_ms, 3),
            "speedup_vs_singles": round(s_ms / g_ms, 2),
            "grouped_device_ms": round(d_ms, 3),
            "grouped_device_gflops": round(flop / 1e9 / (d_ms * 1e-3), 1),
            "note": "step = eager autograd forward + backward from Python (host-bound at "
                    "this size); device = the three grouped launches replayed from graphs"}
        del runners, passes
        del As, Bs, dCs
        out[tag] = rows
    return out


def syrk_report(g, torch, shapes=((8192, 8192), (2048, 2048))):
    """SYRK (lower, trans 'N', beta 0.5, ld = n + 7) on the fused kernel: GFLOP/s counted as
    n(n+1)k (the triangle), with A's panels packed once for both operand roles (policy AUTO)
    and with raw reads only (policy NONE), against the full GEMM of the same shape.  Device
    time, CUDA events, best of a few calls."""
    out = {"note": "uplo L, trans N, beta 0.5, ld = n + 7; flops n(n+1)k; GEMM = the full "
                   "n x n x k product with the same operands"}
    h = g.Handle()
    h.bind_stream()
    for dtype, tag in ((torch.float64, "f64"), (torch.float32, "f32")):
        esz = 8 if tag == "f64" else 4
        rows = {}
        for n, k in shapes:
            A, _, C = make_operands(n + k, dtype, n, n, k)
            lda, ldc = A.stride(1), C.stride(1)
            h.ensure_syrk_workspace("L", "N", n, k, esz)
            h.ensure_workspace("N", "T", n, n, k, esz)

            def best(fn, reps):
                fn()
                torch.cuda.synchronize()
                t = float("inf")
                for _ in range(reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    fn()
                    e1.record()
                    e1.synchronize()
                    t = min(t, e0.elapsed_time(e1))
                return t
            r = {}
            for pol, name in ((g.GFIP_PACK_AUTO, "fused"), (g.GFIP_PACK_NONE, "raw_only")):
                h.set_pack_policy(pol)

                def call():
                    rc = g.gfip_syrk(esz, h.h, "L", "N", n, k, 1.0, A.data_ptr(), lda, 0.5,
                                     C.data_ptr(), ldc)
                    assert rc == 0, rc
                ms = best(call, 2 if n * n * k > 2 ** 36 else 5)
                r[name] = round(n * (n + 1) * k / 1e9 / (ms * 1e-3), 1)
                r[name + "_ms"] = round(ms, 3)
            h.set_pack_policy(g.GFIP_PACK_AUTO)
            gname = g.ENTRY[("fused", esz)]

            def gcall():
                rc = g._gemm_call(gname, h.h, "N", "T", n, n, k, 1.0, A.data_ptr(), lda,
                                  A.data_ptr(), lda, 0.5, C.data_ptr(), ldc)
                assert rc == 0, rc
            gms = best(gcall, 2 if n * n * k > 2 ** 36 else 5)
            r["gemm_ms"] = round(gms, 3)
            r["syrk_time_over_gemm"] = round(r["fused_ms"] / gms, 3)
            peak = FP64_PEAK_GFLOPS if tag == "f64" else FP32_PEAK_GFLOPS
            r["fused_frac_of_peak"] = round(r["fused"] / peak, 4)
            rows[f"{n}x{k}"] = r
            del A, C
        out[tag] = rows
    out["status"] = h.status()
    return out


def trmm_report(g, torch, shapes=((8192, 8192), (2048, 2048))):
    """TRMM (side L, lower, 'N', non-unit, ld = m + 7) on the fused kernel: GFLOP/s counted
    as m(m+1)n (the nonzero products), fused (masked panels packed once) and raw-only,
    against the full GEMM of the same shape.  Device time, CUDA events, best of a few."""
    out = {"note": "side L, uplo L, trans N, diag N, ld = m + 7; flops m(m+1)n; time "
                   "includes the out-of-place product and the copy back into B"}
    h = g.Handle()
    h.bind_stream()
    for dtype, tag in ((torch.float64, "f64"), (torch.float32, "f32")):
        esz = 8 if tag == "f64" else 4
        rows = {}
        for m, n in shapes:
            A, B, C = make_operands(m + n, dtype, m, n, m)
            lda, ldb = A.stride(1), B.stride(1)
            h.ensure_trmm_workspace("L", "L", "N", "N", m, n, esz)
            h.ensure_workspace("N", "N", m, n, m, esz)

            def best(fn, reps):
                fn()
                torch.cuda.synchronize()
                t = float("inf")
                for _ in range(reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    fn()
                    e1.record()
                    e1.synchronize()
                    t = min(t, e0.elapsed_time(e1))
                return t
            reps = 2 if m * m * n > 2 ** 36 else 5
            r = {}
            for pol, name in ((g.GFIP_PACK_AUTO, "fused"), (g.GFIP_PACK_NONE, "raw_only")):
                h.set_pack_policy(pol)

                def call():
                    rc = g.gfip_trmm(esz, h.h, "L", "L", "N", "N", m, n, 1.0, A.data_ptr(), lda,
                                     B.data_ptr(), ldb)
                    assert rc == 0, rc
                ms = best(call, reps)
                r[name] = round(m * (m + 1) * n / 1e9 / (ms * 1e-3), 1)
                r[name + "_ms"] = round(ms, 3)
            h.set_pack_policy(g.GFIP_PACK_AUTO)
            gname = g.ENTRY[("fused", esz)]

            def gcall():
                rc = g._gemm_call(gname, h.h, "N", "N", m, n, m, 1.0, A.data_ptr(), lda,
                                  B.data_ptr(), ldb, 0.0, C.data_ptr(), C.stride(1))
                assert rc == 0, rc
            gms = best(gcall, reps)
            r["gemm_ms"] = round(gms, 3)
            r["trmm_time_over_gemm"] = round(r["fused_ms"] / gms, 3)
            peak = FP64_PEAK_GFLOPS if tag == "f64" else FP32_PEAK_GFLOPS
            r["fused_frac_of_peak"] = round(r["fused"] / peak, 4)
            rows[f"{m}x{n}"] = r
            del A, B, C
        out[tag] = rows
    out["status"] = h.status()
    return out


def trsm_report(g, torch, shapes=((8192, 8192), (2048, 2048))):
    """TRSM (side L, lower, 'N', non-unit, ld = m + 7; a well-conditioned system: off-diagonal
    entries U[-1, 1] / m, diagonal 2) on the fused kernel: GFLOP/s counted as m^2 n (the
    substitution's multiply-adds), fused and raw-only, against the full GEMM of the same
    shape.  Device time of one whole solve (a panel solve and a GEMM update per 512-wide
    panel), CUDA events, best of a few."""
    out = {"note": "side L, uplo L, trans N, diag N, ld = m + 7; flops m^2 n; panels of 512 "
                   "unknowns, each solved in one launch, then one GEMM update"}
    h = g.Handle()
    h.bind_stream()
    for dtype, tag in ((torch.float64, "f64"), (torch.float32, "f32")):
        esz = 8 if tag == "f64" else 4
        rows = {}
        for m, n in shapes:
            A, B, C = make_operands(m + n + 1, dtype, m, n, m)
            A.mul_(1.0 / m)
            A.diagonal().fill_(2.0)
            B0 = B.clone()   # a dense copy (its own layout): only ever copied back into B
            lda, ldb = A.stride(1), B.stride(1)
            h.ensure_trsm_workspace("L", "L", "N", "N", m, n, esz)
            h.ensure_workspace("N", "N", m, n, m, esz)

            def best(fn, reps):
                t = float("inf")
                for _ in range(reps + 1):
                    B.copy_(B0)
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    fn()
                    e1.record()
                    e1.synchronize()
                    t = min(t, e0.elapsed_time(e1))
                return t
            reps = 2 if m * m * n > 2 ** 36 else 5
            r = {}
            for pol, name in ((g.GFIP_PACK_AUTO, "fused"), (g.GFIP_PACK_NONE, "raw_only")):
                h.set_pack_policy(pol)

                def call():
                    rc = g.gfip_trsm(esz, h.h, "L", "L", "N", "N", m, n, 1.0, A.data_ptr(), lda,
                                     B.data_ptr(), ldb)
                    assert rc == 0, rc
                ms = best(call, reps)
                r[name] = round(m * m * n / 1e9 / (ms * 1e-3), 1)
                r[name + "_ms"] = round(ms, 3)
            h.set_pack_policy(g.GFIP_PACK_AUTO)
            gname = g.ENTRY[("fused", esz)]

            def gcall():
                rc = g._gemm_call(gname, h.h, "N", "N", m, n, m, 1.0, A.data_ptr(), lda,
                                  B.data_ptr(), ldb, 0.0, C.data_ptr(), C.stride(1))
                assert rc == 0, rc
            gms = best(gcall, reps)
            r["gemm_ms"] = round(gms, 3)
            r["trsm_time_over_gemm"] = round(r["fused_ms"] / gms, 3)
            peak = FP64_PEAK_GFLOPS if tag == "f64" else FP32_PEAK_GFLOPS
            r["fused_frac_of_peak"] = round(r["fused"] / peak, 4)
            rows[f"{m}x{n}"] = r
            del A, B, B0, C
        out[tag] = rows
    out["status"] = h.status()
    return out


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2302_08417_gb300 import inputs
    oracle.build()
    threads = os.cpu_count() or 1
    rng = np.random.Generator(np.random.PCG64(0))
    lda, ldb, ldc = M + PAD, K + PAD, M + PAD
    A = inputs.colmajor(rng, M, K, lda)
    cols = 2 * threads
    B = inputs.colmajor(rng, K, cols, ldb)
    C = inputs.colmajor(rng, M, cols, ldc)

    def step():
        Cs = C.copy()
        rc = oracle.gemm("N", "N", M, cols, K, ALPHA, A, lda, B, ldb, BETA, Cs, ldc,
                         nthreads=threads)
        assert rc == 0
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    val = gflop(M, cols, K) / dt
    sample = (f"each step: the first {cols} of {N} columns of C (m=k={M}, lda=ldb=ldc={M+PAD},"
              f" alpha=1, beta=0.5), FP64 j-p-i triple loop, OpenMP over columns")
    # the metric and config of this arm are those of the GPU arm on the same arguments
    print(json.dumps({
        "impl": "reference", "metric": f"{args.dtype} gemm throughput ({args.variant})",
        "value": round(val, 3),
        "unit": "GFLOP/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": M, "n": N, "k": K, "transa": "N", "transb": "N",
                   "lda": lda, "ldb": ldb, "ldc": ldc, "alpha": ALPHA, "beta": BETA,
                   "parallelism": f"host cores x{threads}"},
        "cpu_baseline": {"value": round(val, 3), "unit": "GFLOP/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(val, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def compact_summary(result) -> dict:
    """The figures a reader needs first, small enough to survive a truncated log tail: per
    size, [fused GFLOP/s, fused / best plain variant, noise band] in both dtypes, and the
    headline of each extension report."""
    out = {}
    fvp = result.get("fip_vs_plain")
    if fvp:
        for tag in ("f64", "f32"):
            out[f"{tag}_n:[fused_gflops,fused/best_plain,noise]"] = {
                n: [r["gflops"]["fused"], r["fused_over_best_plain"], r["noise"]]
                for n, r in fvp[tag].items()}
        out["extra:[fused/best_plain,noise]"] = {
            k: [r["fused_over_best_plain"], r["noise"]] for k, r in fvp["extra"].items()}
        out["min_fused/best_plain-noise"] = round(min(
            r["fused_over_best_plain"] + r["noise"]
            for tag in ("f64", "f32") for r in fvp[tag].values()) - 1.0, 4)
    if "roofline_f32" in result:
        out["f32_8192_frac_of_ffma_peak"] = result["roofline_f32"]["frac"]
    emu = result.get("emulated_fp64")
    if emu:
        out["emulated_fp64_8192:[S:tflops,max_rel_err_uniform,logmag]"] = {
            k[len("slices_"):]: [round(v["gflops"] / 1e3, 1), v["max_rel_err"],
                                 emu["logmag"][k]["max_rel_err"]]
            for k, v in emu.get("uniform", {}).items()}
    bat = result.get("batched")
    if bat:
        out["batched_4096:[grouped_gflops,frac_of_peak,x_singles]"] = {
            tag: [v["grouped_graph_gflops"],
                  round(v["grouped_graph_gflops"] /
                        (FP64_PEAK_GFLOPS if tag == "f64" else FP32_PEAK_GFLOPS), 4),
                  v["speedup_vs_singles_graph"]]
            for tag, v in bat.items() if isinstance(v, dict) and "grouped_graph_gflops" in v}
    ag = result.get("autograd")
    if ag:
        out["autograd:[fused_gflops,x_cublas]"] = {
            f"{tag} {shape}": [v["fused"], v["fused_over_cublas"]]
            for tag in ("f64", "f32") for shape, v in ag.get(tag, {}).items()
            if "fused" in v}
    ts = result.get("trsm")
    if ts:
        out["trsm:[fused_gflops,time_over_gemm]"] = {
            f"{tag} {shape}": [v["fused"], v["trsm_time_over_gemm"]]
            for tag in ("f64", "f32") for shape, v in ts.get(tag, {}).items()
            if "fused" in v}
    return out


def main():
    global M, N, K, WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-spectrum", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-emulation", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--size", type=int, default=M, help="m = n = k (default: the headline)")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    ap.add_argument("--variant", default="fused", choices=["fused", "direct",
                                                          "pack_then_compute"])
    ap.add_argument("--sweep", default=None, metavar="SIZES",
                    help="only run the fused-vs-plain size sweep: 'all' (16 .. 16384) or a "
                         "comma-separated list of sizes; prints one JSON line")
    ap.add_argument("--sweep-dtypes", default="f64,f32")
    ap.add_argument("--sweep-md", default=None, help="also write the sweep as a markdown table")
    ap.add_argument("--emulation-only", type=int, default=0, metavar="N",
                    help="only run the emulated-FP64 report at m = n = k = N")
    ap.add_argument("--slices", default="3,5,7,9", help="digit counts of the emulated report")
    ap.add_argument("--batched-only", type=int, default=0, metavar="COUNT",
                    help="only run the grouped-GEMM report on COUNT problems")
    ap.add_argument("--autograd-only", action="store_true",
                    help="only run the differentiable-GEMM report")
    ap.add_argument("--trsm-only", type=int, default=0, metavar="N",
                    help="only the TRSM report, on an N x N system with N right-hand sides")
    ap.add_argument("--syrk-only", action="store_true",
                    help="only run the SYRK, TRMM and TRSM reports")
    ap.add_argument("--no-syrk", action="store_true",
                    help="skip the SYRK, TRMM and TRSM reports")
    ap.add_argument("--no-autograd", action="store_true")
    args = ap.parse_args()
    if args.size != M or args.dtype != "f64" or args.variant != "fused":
        M = N = K = args.size
        WORKLOAD = workload(args.dtype, M, args.variant)
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    barrier(world)
    from paper_2302_08417_gb300 import gemmfip as g

    torch.cuda.set_device(local)
    h = g.Handle()
    h.bind_stream()
    stream = torch.cuda.current_stream()
    if (args.emulation_only or args.batched_only or args.autograd_only or args.syrk_only
            or args.trsm_only):
        out = {}
        if args.trsm_only:
            out["trsm"] = trsm_report(g, torch, shapes=((args.trsm_only, args.trsm_only),))
        if args.syrk_only:
            out["syrk"] = syrk_report(g, torch)
            out["trmm"] = trmm_report(g, torch)
            out["trsm"] = trsm_report(g, torch)
        if args.autograd_only:
            out["autograd"] = autograd_report(torch)
        if args.emulation_only:
            out["emulated_fp64"] = emulation_report(
                h, g, torch, n=args.emulation_only,
                slice_counts=tuple(int(x) for x in args.slices.split(",")))
        if args.batched_only:
            out["batched"] = batched_report(g, torch, count=args.batched_only)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    if args.sweep is not None:
        from paper_2302_08417_gb300 import inputs
        sizes = (inputs.config_sizes() if args.sweep == "all"
                 else [int(x) for x in args.sweep.split(",")])
        clocks = ClockSampler(local)
        clocks.start()
        res = sweep(h, g, torch, sizes, tuple(args.sweep_dtypes.split(",")))
        res["clocks"] = clocks.stop()
        if rank == 0:
            print(json.dumps({"sweep": res}), flush=True)
            if args.sweep_md:
                with open(args.sweep_md, "w") as f:
                    f.write(sweep_markdown(res))
        return
    f64 = args.dtype == "f64"
    esz = 8 if f64 else 4
    A, B, C = make_operands(1234 + rank, torch.float64 if f64 else torch.float32)
    lda, ldb, ldc = A.stride(1), B.stride(1), C.stride(1)
    h.ensure_workspace("N", "N", M, N, K, esz)
    entry = g.ENTRY[(args.variant, esz)]

    def step():
        rc = g._gemm_call(entry, h.h, "N", "N", M, N, K, ALPHA, A.data_ptr(), lda,
                          B.data_ptr(), ldb, BETA, C.data_ptr(), ldc)
        if rc != 0:
            raise g.GemmError(rc, entry)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches_per_step, grid = g.gfip_last_launch_info(h.h)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)
    barrier(world)
    torch.cuda.synchronize()
    events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for e0, e1 in events:
        e0.record(stream)
        step()
        e1.record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    per_launch_ms = [e0.elapsed_time(e1) for e0, e1 in events]
    total_ms = max_over_ranks(world, total_ms)
    status = h.status()

    value = world * args.steps * gflop() / (total_ms * 1e-3)
    avg_launch_s = sum(per_launch_ms) / len(per_launch_ms) * 1e-3
    achieved = gflop() / avg_launch_s
    th = kernel_hash()
    headline = (M == 8192 and f64 and args.variant == "fused")
    traffic = (TRAFFIC["bytes_per_launch"]
               if headline and TRAFFIC["kernel_hash"] == th else None)
    peak = FP64_PEAK_GFLOPS if f64 else FP32_PEAK_GFLOPS

    result = {
        "metric": f"{args.dtype} gemm throughput ({args.variant})", "value": round(value, 2),
        "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": M, "n": N, "k": K, "transa": "N", "transb": "N",
                   "lda": lda, "ldb": ldb, "ldc": ldc, "alpha": ALPHA, "beta": BETA,
                   "l2": f"inputs larger than L2 ({3 * A.stride(1) * A.shape[1] * esz / 1e9:.2f}"
                         " GB of operands vs 0.136 GB L2), no flush",
                   "parallelism": f"replicas x{world}", "grid": grid},
        "roofline": {"bound": "alu", "achieved": round(achieved, 2),
                     "peak": round(peak, 1), "unit": "GFLOP/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "kernel": f"gfip::gemm_kernel<{'double' if f64 else 'float'}>",
                     "peak_basis": ("152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (DFMA rate "
                                    "measured by peak_probe)" if f64 else
                                    "152 SMs x 128 FFMA/clk x 2 flop x 2070 MHz"),
                     "hbm_floor_ms": round(algorithmic_bytes(s=esz) / HBM_GBS / 1e6, 3)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "device_status": status,
    }

    if rank == 0 and not args.no_cpu:
        # end to end through the public API with pinned host buffers
        hA, bufA = host_copy(A)
        hB, bufB = host_copy(B)
        hC, bufC = host_copy(C)
        from paper_2302_08417_gb300 import gemm as pub_gemm
        pub_gemm(hA, hB, hC, ALPHA, BETA, variant=args.variant, handle=h)   # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            pub_gemm(hA, hB, hC, ALPHA, BETA, variant=args.variant, handle=h)
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        result["e2e"] = {"value": round(gflop() / e2e_s, 2), "unit": "GFLOP/s",
                         "h2d_bytes_per_step": g.span_bytes(hA) + g.span_bytes(hB)
                         + g.span_bytes(hC),
                         "d2h_bytes_per_step": g.span_bytes(hC),
                         "steps": args.e2e_steps,
                         "path": "paper_2302_08417_gb300.gemm(pinned host tensors) -> "
                                 f"{entry} per 1024-column block of C, uploads, blocks and "
                                 "downloads pipelined on three streams; copies and compute "
                                 "inside the timed region"}
        # oracle on the host cores, bounded sample of the same workload
        result["cpu_baseline"] = cpu_oracle_sample(
            bufA.numpy().reshape(-1), bufB.numpy().reshape(-1), bufC.numpy().reshape(-1),
            M, K, lda, ldb, ldc)
        result["cpu_baseline"]["single_thread"] = oracle_single_thread()
    if rank == 0 and not args.no_emulation:
        result["emulated_fp64"] = emulation_report(
            h, g, torch, slice_counts=tuple(int(x) for x in args.slices.split(",")))
    if rank == 0 and not args.no_batched:
        result["batched"] = batched_report(g, torch)
    if rank == 0 and not args.no_autograd:
        result["autograd"] = autograd_report(torch)
    if rank == 0 and not args.no_syrk:
        result["syrk"] = syrk_report(g, torch)
        result["trmm"] = trmm_report(g, torch)
        result["trsm"] = trsm_report(g, torch)
    if rank == 0 and not args.no_spectrum:
        from paper_2302_08417_gb300 import inputs
        clk = ClockSampler(local)
        clk.start()
        result["fip_vs_plain"] = sweep(h, g, torch, inputs.config_sizes())
        result["fip_vs_plain"]["extra"] = extra_cases(h, g, torch)
        result["fip_vs_plain"]["clocks"] = clk.stop()
        f32 = result["fip_vs_plain"]["f32"][str(8192)]
        result["roofline_f32"] = {
            "bound": "alu", "achieved": f32["gflops"]["fused"], "peak": round(FP32_PEAK_GFLOPS, 1),
            "unit": "GFLOP/s", "frac": f32["frac"], "traffic": None,
            "kernel": "gfip::ws::ws_gemm_kernel (FP32, warp-specialised)",
            "workload": workload("f32", 8192),
            "peak_basis": "152 SMs x 128 FFMA/clk x 2 flop x 2070 MHz"}
    if rank == 0:
        result["summary"] = compact_summary(result)
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
