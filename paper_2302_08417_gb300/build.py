"""Builds the CUDA library in-tree: paper_2302_08417_gb300/_build/libgemmfip.so.

Every translation unit is compiled for sm_103a only, in parallel, then linked against the
shared CUDA runtime (so the process shares one runtime with PyTorch).  Also builds the
stand-alone peak probe used to measure the FP64/FP32 arithmetic roofline.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libgemmfip.so")
PROBE = os.path.join(OUT, "peak_probe")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
LIB_SOURCES = ["gfip_api.cu", "gfip_f64.cu", "gfip_f32.cu", "gfip_f32_ws.cu", "gfip_f64_tmask.cu",
               "gfip_f32_tmask.cu", "gfip_ozaki.cu", "gfip_grouped.cu", "gfip_trsm.cu"]
HEADERS = ["gfip_internal.h", "gfip_kernels.cuh", "gfip_ws.cuh", "gfip_grouped.h",
           "gfip_testing.h"]
NVCC_FLAGS = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                     "-I" + os.path.join(ROOT, "include")]
# Extra nvcc arguments (e.g. "-DGFIP_F32_UNROLL=16" to override a tile parameter of
# gfip_internal.h); a build with them is forced, since the sources did not change.
EXTRA_FLAGS = os.environ.get("GFIP_NVCC_EXTRA", "").split()


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build")
    return path


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd: list[str]) -> None:
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")


def build(force: bool = False, probe: bool = True, verbose: bool = False) -> str:
    """Compile (if stale) and return the path of libgemmfip.so."""
    os.makedirs(OUT, exist_ok=True)
    force = force or bool(EXTRA_FLAGS)
    cc = nvcc()
    headers = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include",
                                                                       "gemmfip.h")]
    jobs = []
    objs = []
    for src in LIB_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            extra = ["-Xptxas", "-v"] if verbose else []
            jobs.append([cc] + NVCC_FLAGS + EXTRA_FLAGS + extra + ["-c", s, "-o", o])
    if probe:
        ps = os.path.join(CSRC, "peak_probe.cu")
        if force or _stale(PROBE, [ps]):
            jobs.append([cc] + ARCH + ["-O3", "-std=c++17", ps, "-o", PROBE])
    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        list(ex.map(_run, jobs))
    if force or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        _run([cc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
