"""Python binding of the C ABI in include/gemmfip.h (argument marshalling only).

The functions ``gfip_*`` below have the names and argument order of the C entry points and
take plain integers for device pointers and streams; every step of the GEMM runs in the CUDA
library.  :class:`Handle` and :func:`gemm` add PyTorch conveniences on top: the workspace is
a caller-owned ``torch.uint8`` CUDA tensor, the stream is torch's current stream, and
matrices are 2-D column-major tensor views (``X.stride(0) == 1``, leading dimension
``X.stride(1)``), exactly the storage a BLAS caller passes.

There is no fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgemmfip.so")

GFIP_OK = 0
GFIP_ERR_HANDLE = 1
GFIP_ERR_CUDA = 2
GFIP_ERR_WORKSPACE = 3
GFIP_ERR_NULLPTR = 4
GFIP_ERR_DEVICE = 5
GFIP_ERR_SIZE = 6
GFIP_ERR_ARG = 7
GFIP_ERR_SCRATCH_LIMIT = 8
GFIP_ERR_CAPTURE = 9
GFIP_NOALLOC_SCRATCH_BYTES = 64 * 1024 * 1024
GFIP_STATUS_BAD_SEGMENT = 0x1
GFIP_STATUS_MMA_TIMEOUT = 0x2
GFIP_STATUS_BAD_PROBLEM = 0x4
GFIP_STATUS_WAIT_TIMEOUT = 0x8
GFIP_GROUP_TILE_DEFAULT, GFIP_GROUP_TILE_SMALL, GFIP_GROUP_TILE_TINY = 0, 1, 2
GFIP_GROUP_TILE_16X8, GFIP_GROUP_TILE_8X16 = 3, 4


def GFIP_GROUP_PLAN(tile: int, splits: int) -> int:
    return tile | (splits << 8)

GFIP_PACK_AUTO, GFIP_PACK_NONE, GFIP_PACK_A, GFIP_PACK_B, GFIP_PACK_BOTH = range(5)
GFIP_PACKER_AUTO, GFIP_PACKER_LINE, GFIP_PACKER_SHARED = range(3)

# exported symbol -> (restype, argtypes)
_i64, _dbl, _flt, _ptr = ctypes.c_int64, ctypes.c_double, ctypes.c_float, ctypes.c_void_p
_chr, _int, _sz = ctypes.c_char, ctypes.c_int, ctypes.c_size_t
_GEMM_D = [_ptr, _chr, _chr, _i64, _i64, _i64, _dbl, _ptr, _i64, _ptr, _i64, _dbl, _ptr, _i64]
_GEMM_S = [_ptr, _chr, _chr, _i64, _i64, _i64, _flt, _ptr, _i64, _ptr, _i64, _flt, _ptr, _i64]
SIGNATURES = {
    "gfip_create": (_int, [ctypes.POINTER(_ptr)]),
    "gfip_destroy": (_int, [_ptr]),
    "gfip_set_stream": (_int, [_ptr, _ptr]),
    "gfip_workspace_size": (_sz, [_ptr, _chr, _chr, _i64, _i64, _i64, _int]),
    "gfip_set_workspace": (_int, [_ptr, _ptr, _sz]),
    "gfip_set_pack_policy": (_int, [_ptr, _int]),
    "gfip_set_packer": (_int, [_ptr, _int]),
    "gfip_dgemm": (_int, _GEMM_D),
    "gfip_sgemm": (_int, _GEMM_S),
    "gfip_dgemm_direct": (_int, _GEMM_D),
    "gfip_sgemm_direct": (_int, _GEMM_S),
    "gfip_dgemm_pack_then_compute": (_int, _GEMM_D),
    "gfip_sgemm_pack_then_compute": (_int, _GEMM_S),
    "gfip_get_status": (_int, [_ptr, ctypes.POINTER(ctypes.c_uint32)]),
    "gfip_last_launch_info": (_int, [_ptr, ctypes.POINTER(_int), ctypes.POINTER(_int)]),
    "gfip_error_string": (ctypes.c_char_p, [_int]),
    "gfip_dgemm_noalloc": (_int, [_chr, _chr, _i64, _i64, _i64, _dbl, _ptr, _i64, _ptr, _i64,
                                  _dbl, _ptr, _i64, _ptr]),
    "gfip_ozaki_workspace_size": (_sz, [_ptr, _i64, _i64, _i64, _int]),
    "gfip_grouped_workspace_size": (_sz, [_ptr, _int]),
    "gfip_dgemm_grouped": (_int, [_ptr, _int] + [_ptr] * 13 + [_int]),
    "gfip_sgemm_grouped": (_int, [_ptr, _int] + [_ptr] * 13 + [_int]),
    "gfip_grouped_plan_workspace_size": (_sz, [_ptr, _int, _i64, _int]),
    "gfip_dgemm_grouped_plan": (_int, [_ptr, _int] + [_ptr] * 15 + [_i64]),
    "gfip_sgemm_grouped_plan": (_int, [_ptr, _int] + [_ptr] * 15 + [_i64]),
    "gfip_dgemm_ozaki": (_int, _GEMM_D + [_int]),
    "gfip_debug_ozaki_timeout": (_int, [_ptr, _int, ctypes.c_uint64]),
    "gfip_syrk_workspace_size": (_sz, [_ptr, _chr, _chr, _i64, _i64, _int]),
    "gfip_dsyrk": (_int, [_ptr, _chr, _chr, _i64, _i64, _dbl, _ptr, _i64, _dbl, _ptr, _i64]),
    "gfip_ssyrk": (_int, [_ptr, _chr, _chr, _i64, _i64, _flt, _ptr, _i64, _flt, _ptr, _i64]),
    "gfip_trmm_workspace_size": (_sz, [_ptr, _chr, _chr, _chr, _chr, _i64, _i64, _int]),
    "gfip_dtrmm": (_int, [_ptr, _chr, _chr, _chr, _chr, _i64, _i64, _dbl, _ptr, _i64, _ptr,
                          _i64]),
    "gfip_strmm": (_int, [_ptr, _chr, _chr, _chr, _chr, _i64, _i64, _flt, _ptr, _i64, _ptr,
                          _i64]),
    "gfip_trsm_workspace_size": (_sz, [_ptr, _chr, _chr, _chr, _chr, _i64, _i64, _int]),
    "gfip_dtrsm": (_int, [_ptr, _chr, _chr, _chr, _chr, _i64, _i64, _dbl, _ptr, _i64, _ptr,
                          _i64]),
    "gfip_strsm": (_int, [_ptr, _chr, _chr, _chr, _chr, _i64, _i64, _flt, _ptr, _i64, _ptr,
                          _i64]),
}

_lock = threading.Lock()
_lib = None


class GemmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {error_string(code)} (code {code})")


def load(path: str = LIB_PATH):
    """Loads libgemmfip.so (built by ``paper_2302_08417_gb300.build``); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(
                    f"{path} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def error_string(code: int) -> str:
    return load().gfip_error_string(code).decode()


def _b(c: str) -> bytes:
    return c.encode() if isinstance(c, str) else c


# ---- thin wrappers with the C names (pointers and streams are ints) -------------------

def gfip_create() -> int:
    h = _ptr()
    rc = load().gfip_create(ctypes.byref(h))
    if rc != GFIP_OK:
        raise GemmError(rc, "gfip_create")
    return h.value


def gfip_destroy(handle: int) -> int:
    return load().gfip_destroy(handle)


def gfip_set_stream(handle: int, stream: int) -> int:
    return load().gfip_set_stream(handle, stream or None)


def gfip_workspace_size(handle, transa, transb, m, n, k, elem_bytes) -> int:
    return load().gfip_workspace_size(handle, _b(transa), _b(transb), m, n, k, elem_bytes)


def gfip_set_workspace(handle: int, ptr: int, nbytes: int) -> int:
    return load().gfip_set_workspace(handle, ptr or None, nbytes)


def gfip_set_pack_policy(handle: int, policy: int) -> int:
    return load().gfip_set_pack_policy(handle, policy)


def gfip_set_packer(handle: int, packer: int) -> int:
    return load().gfip_set_packer(handle, packer)


def _gemm_call(name, handle, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc):
    fn = getattr(load(), name)
    return fn(handle, _b(transa), _b(transb), m, n, k, alpha, A or None, lda, B or None, ldb,
              beta, C or None, ldc)


def gfip_dgemm(*a):
    return _gemm_call("gfip_dgemm", *a)


def gfip_sgemm(*a):
    return _gemm_call("gfip_sgemm", *a)


def gfip_dgemm_direct(*a):
    return _gemm_call("gfip_dgemm_direct", *a)


def gfip_sgemm_direct(*a):
    return _gemm_call("gfip_sgemm_direct", *a)


def gfip_dgemm_pack_then_compute(*a):
    return _gemm_call("gfip_dgemm_pack_then_compute", *a)


def gfip_sgemm_pack_then_compute(*a):
    return _gemm_call("gfip_sgemm_pack_then_compute", *a)


def gfip_get_status(handle: int) -> int:
    v = ctypes.c_uint32(0)
    rc = load().gfip_get_status(handle, ctypes.byref(v))
    if rc != GFIP_OK:
        raise GemmError(rc, "gfip_get_status")
    return int(v.value)


def gfip_last_launch_info(handle: int) -> tuple[int, int]:
    a, b = _int(0), _int(0)
    load().gfip_last_launch_info(handle, ctypes.byref(a), ctypes.byref(b))
    return int(a.value), int(b.value)


def gfip_dgemm_noalloc(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                       stream=0) -> int:
    """The allocation-free FP64 entry point: BLAS dgemm arguments plus a stream, no handle and
    no workspace; its scratch is a fixed static device array inside the library."""
    return load().gfip_dgemm_noalloc(_b(transa), _b(transb), m, n, k, alpha, A or None, lda,
                                     B or None, ldb, beta, C or None, ldc, stream or None)


def gfip_ozaki_workspace_size(handle, m, n, k, slices) -> int:
    return load().gfip_ozaki_workspace_size(handle, m, n, k, slices)


def gfip_dgemm_ozaki(handle, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                     slices) -> int:
    """FP64 GEMM emulated with exact BF16 digit products on the tensor cores."""
    return load().gfip_dgemm_ozaki(handle, _b(transa), _b(transb), m, n, k, alpha, A or None,
                                   lda, B or None, ldb, beta, C or None, ldc, slices)


def gfip_debug_ozaki_timeout(handle, enable: bool, wait_ns: int = 0) -> int:
    """Test hook: later gfip_dgemm_ozaki calls withhold one operand copy in the first CTA so
    that its bounded wait (wait_ns; 0 = the 2 s default) runs out."""
    return load().gfip_debug_ozaki_timeout(handle, int(bool(enable)), int(wait_ns))


def gfip_syrk_workspace_size(handle, uplo, trans, n, k, elem_bytes) -> int:
    return load().gfip_syrk_workspace_size(handle, _b(uplo), _b(trans), n, k, elem_bytes)


def gfip_syrk(esz, handle, uplo, trans, n, k, alpha, A, lda, beta, C, ldc) -> int:
    """gfip_dsyrk (esz 8) or gfip_ssyrk (esz 4); A and C are device pointers."""
    fn = load().gfip_dsyrk if esz == 8 else load().gfip_ssyrk
    return fn(handle, _b(uplo), _b(trans), n, k, alpha, A or None, lda, beta, C or None, ldc)


def gfip_trmm_workspace_size(handle, side, uplo, transa, diag, m, n, elem_bytes) -> int:
    return load().gfip_trmm_workspace_size(handle, _b(side), _b(uplo), _b(transa), _b(diag), m,
                                           n, elem_bytes)


def gfip_trmm(esz, handle, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb) -> int:
    """gfip_dtrmm (esz 8) or gfip_strmm (esz 4); A and B are device pointers."""
    fn = load().gfip_dtrmm if esz == 8 else load().gfip_strmm
    return fn(handle, _b(side), _b(uplo), _b(transa), _b(diag), m, n, alpha, A or None, lda,
              B or None, ldb)


def gfip_trsm_workspace_size(handle, side, uplo, transa, diag, m, n, elem_bytes) -> int:
    return load().gfip_trsm_workspace_size(handle, _b(side), _b(uplo), _b(transa), _b(diag), m,
                                           n, elem_bytes)


def gfip_trsm(esz, handle, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb) -> int:
    """gfip_dtrsm (esz 8) or gfip_strsm (esz 4); A and B are device pointers."""
    fn = load().gfip_dtrsm if esz == 8 else load().gfip_strsm
    return fn(handle, _b(side), _b(uplo), _b(transa), _b(diag), m, n, alpha, A or None, lda,
              B or None, ldb)


def gfip_grouped_workspace_size(handle, count) -> int:
    return load().gfip_grouped_workspace_size(handle, count)


def gfip_gemm_grouped(esz, handle, count, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta,
                      C, ldc, tile) -> int:
    """Grouped GEMM; every array argument is a device pointer (int)."""
    fn = load().gfip_dgemm_grouped if esz == 8 else load().gfip_sgemm_grouped
    return fn(handle, count, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, tile)


def gfip_grouped_plan_workspace_size(handle, count, split_elems, elem_bytes) -> int:
    return load().gfip_grouped_plan_workspace_size(handle, count, split_elems, elem_bytes)


def gfip_gemm_grouped_plan(esz, handle, count, transa, transb, m, n, k, alpha, A, lda, B, ldb,
                           beta, C, ldc, plan, order, split_elems) -> int:
    """Grouped GEMM with a per-problem plan; array arguments are device pointers (int)."""
    fn = load().gfip_dgemm_grouped_plan if esz == 8 else load().gfip_sgemm_grouped_plan
    return fn(handle, count, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, plan,
              order or None, split_elems)


ENTRY = {
    ("fused", 8): "gfip_dgemm", ("fused", 4): "gfip_sgemm",
    ("direct", 8): "gfip_dgemm_direct", ("direct", 4): "gfip_sgemm_direct",
    ("pack_then_compute", 8): "gfip_dgemm_pack_then_compute",
    ("pack_then_compute", 4): "gfip_sgemm_pack_then_compute",
}


# ---- PyTorch conveniences -------------------------------------------------------------

class Handle:
    """A library handle bound to the current CUDA device, with a torch-allocated workspace
    that grows on demand (the library itself never allocates)."""

    def __init__(self, workspace_bytes: int = 0):
        import torch
        self._torch = torch
        self.h = gfip_create()
        self.workspace = None
        self.stream = None
        if workspace_bytes:
            self._set_ws(workspace_bytes)

    def _set_ws(self, nbytes: int):
        torch = self._torch
        self.workspace = torch.empty(max(nbytes, 16), dtype=torch.uint8, device="cuda")
        rc = gfip_set_workspace(self.h, self.workspace.data_ptr(), self.workspace.numel())
        if rc != GFIP_OK:
            raise GemmError(rc, "gfip_set_workspace")

    def ensure_workspace(self, transa, transb, m, n, k, elem_bytes):
        need = gfip_workspace_size(self.h, transa, transb, m, n, k, elem_bytes)
        if self.workspace is None or self.workspace.numel() < need:
            if self.workspace is not None:
                self._torch.cuda.current_stream().synchronize()
            self._set_ws(int(need * 1.25) + (1 << 20))

    def ensure_syrk_workspace(self, uplo, trans, n, k, elem_bytes):
        need = gfip_syrk_workspace_size(self.h, uplo, trans, n, k, elem_bytes)
        if self.workspace is None or self.workspace.numel() < need:
            if self.workspace is not None:
                self._torch.cuda.current_stream().synchronize()
            self._set_ws(int(need * 1.25) + (1 << 20))

    def ensure_trmm_workspace(self, side, uplo, transa, diag, m, n, elem_bytes):
        need = gfip_trmm_workspace_size(self.h, side, uplo, transa, diag, m, n, elem_bytes)
        if self.workspace is None or self.workspace.numel() < need:
            if self.workspace is not None:
                self._torch.cuda.current_stream().synchronize()
            self._set_ws(int(need * 1.25) + (1 << 20))

    def ensure_trsm_workspace(self, side, uplo, transa, diag, m, n, elem_bytes):
        need = gfip_trsm_workspace_size(self.h, side, uplo, transa, diag, m, n, elem_bytes)
        if self.workspace is None or self.workspace.numel() < need:
            if self.workspace is not None:
                self._torch.cuda.current_stream().synchronize()
            self._set_ws(int(need * 1.25) + (1 << 20))

    def bind_stream(self, stream=None):
        torch = self._torch
        s = stream if stream is not None else torch.cuda.current_stream()
        if self.stream != s.cuda_stream:
            rc = gfip_set_stream(self.h, s.cuda_stream)
            if rc != GFIP_OK:
                raise GemmError(rc, "gfip_set_stream")
            self.stream = s.cuda_stream

    def ensure_ozaki_workspace(self, m, n, k, slices):
        need = gfip_ozaki_workspace_size(self.h, m, n, k, slices)
        if self.workspace is None or self.workspace.numel() < need:
            if self.workspace is not None:
                self._torch.cuda.current_stream().synchronize()
            self._set_ws(int(need * 1.1) + (1 << 20))

    def set_pack_policy(self, policy: int):
        rc = gfip_set_pack_policy(self.h, policy)
        if rc != GFIP_OK:
            raise GemmError(rc, "gfip_set_pack_policy")

    def set_packer(self, packer: int):
        rc = gfip_set_packer(self.h, packer)
        if rc != GFIP_OK:
            raise GemmError(rc, "gfip_set_packer")

    def status(self) -> int:
        return gfip_get_status(self.h)

    def close(self):
        if self.h:
            gfip_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default: dict = {}


def default_handle() -> Handle:
    import torch
    dev = torch.cuda.current_device()
    if dev not in _default:
        _default[dev] = Handle()
    return _default[dev]


def _colmajor_ld(X, name):
    if X.dim() != 2:
        raise ValueError(f"{name} must be a 2-D column-major view")
    rows, cols = X.shape
    if rows > 1 and X.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1); pass X.t() of a "
                         "row-major tensor, or X.t().contiguous().t()")
    ld = X.stride(1) if cols > 1 else max(rows, 1)
    return max(ld, rows, 1)


def _span(X):
    """1-D view of the storage a column-major 2-D view X occupies."""
    import torch
    rows, cols = X.shape
    ld = _colmajor_ld(X, "matrix")
    n = ld * (cols - 1) + rows if rows and cols else 0
    return torch.as_strided(X, (n,), (1,))


def span_bytes(X) -> int:
    return _span(X).numel() * X.element_size()


def _span_to_device(X):
    import torch
    rows, cols = X.shape
    ld = _colmajor_ld(X, "matrix")
    flat = _span(X).to(torch.device("cuda", torch.cuda.current_device()), non_blocking=True)
    if flat.numel() == 0:
        return torch.empty((rows, cols), dtype=X.dtype, device=flat.device)
    return torch.as_strided(flat, (rows, cols), (1, ld))


# Column blocks of C in the pipelined host path: none below this many columns of C.
HOST_BLOCK_COLS = 1024


def host_blocks(n: int, transb: str) -> list[tuple[int, int]]:
    """Column ranges [j0, j1) of C that the end-to-end path runs as separate calls: n //
    HOST_BLOCK_COLS near-equal blocks (each at least HOST_BLOCK_COLS wide) when op(B) = B,
    else (or below two blocks) one range.  An empty C gives one empty range."""
    blocks = n // HOST_BLOCK_COLS if transb.upper() == "N" else 1
    if blocks < 2:
        return [(0, n)]
    bounds = [n * q // blocks for q in range(blocks + 1)]
    return list(zip(bounds[:-1], bounds[1:]))


def _gemm_host(A, B, C_h, alpha, beta, transa, transb, variant, handle):
    """The end-to-end path: host operands in, host result out.  Each operand's storage span
    (ld*(cols-1) + rows elements) is copied as is, so leading dimensions are kept.

    With op(B) = B ('N') and at least two blocks of HOST_BLOCK_COLS columns, the product runs
    as a pipeline over column blocks of C: A goes up first, then block q's columns of B (and
    of C unless beta == 0 and ldc == m) go up on a copy stream while block q-1 computes, and
    block q's result comes down on another stream while block q+1 computes; every block is
    one call of the library on the device.  (Results equal the single device call's within
    the bound; the blocks' schedules differ, so not necessarily bit for bit.)  Otherwise:
    copy all, one call, copy back."""
    import torch
    n = C_h.shape[1]
    ranges = host_blocks(n, transb)
    if len(ranges) < 2 or C_h.shape[0] == 0 or B.shape[0] == 0:
        dA, dB, dC = (_span_to_device(X) for X in (A, B, C_h))
        gemm(dA, dB, dC, alpha, beta, transa, transb, variant, handle)
        _span(C_h).copy_(_span(dC), non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return C_h
    dev = torch.device("cuda", torch.cuda.current_device())
    compute = torch.cuda.current_stream()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    s_in.wait_stream(compute)     # device buffers below are allocated on `compute`
    spanB, spanC = _span(B), _span(C_h)
    dB_flat = torch.empty(spanB.numel(), dtype=B.dtype, device=dev)
    dC_flat = torch.empty(spanC.numel(), dtype=C_h.dtype, device=dev)
    ldb, ldc = _colmajor_ld(B, "B"), _colmajor_ld(C_h, "C")
    k, m = B.shape[0], C_h.shape[0]
    # C goes up when beta reads it, or when its rows m..ldc-1 lie inside a block's span
    # (they travel up and back down unchanged)
    upload_c = beta != 0.0 or ldc > m
    with torch.cuda.stream(s_in):
        dA = _span_to_device(A)
        ins = []
        for j0, j1 in ranges:
            b0, b1 = j0 * ldb, (j1 - 1) * ldb + k
            dB_flat[b0:b1].copy_(spanB[b0:b1], non_blocking=True)
            if upload_c:
                c0, c1 = j0 * ldc, (j1 - 1) * ldc + m
                dC_flat[c0:c1].copy_(spanC[c0:c1], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s_in)
            ins.append(ev)
    for q, (j0, j1) in enumerate(ranges):
        compute.wait_event(ins[q])
        dBq = torch.as_strided(dB_flat, (k, j1 - j0), (1, ldb), j0 * ldb)
        dCq = torch.as_strided(dC_flat, (m, j1 - j0), (1, ldc), j0 * ldc)
        gemm(dA, dBq, dCq, alpha, beta, transa, "N", variant, handle)
        done = torch.cuda.Event()
        done.record(compute)
        s_out.wait_event(done)
        with torch.cuda.stream(s_out):
            c0, c1 = j0 * ldc, (j1 - 1) * ldc + m
            spanC[c0:c1].copy_(dC_flat[c0:c1], non_blocking=True)
    # the last download waits on the last block, which waits on every upload: once it is
    # done, no stream still uses the device buffers
    s_out.synchronize()
    return C_h


def gemm(A, B, C=None, alpha: float = 1.0, beta: float = 0.0, transa: str = "N",
         transb: str = "N", variant: str = "fused", handle: Handle | None = None):
    """``C := alpha*op(A)*op(B) + beta*C`` on column-major 2-D tensors (float64 or float32).

    A and B are the STORED matrices (A is m x k for transa 'N', k x m for 'T'); C is m x n
    and updated in place (allocated when None, then beta must be 0).  CUDA tensors run
    asynchronously on torch's current stream.  CPU tensors are copied to the GPU, computed,
    and the result copied back into C (the end-to-end path); pinned memory makes the copies
    asynchronous.  Returns C."""
    import torch
    host = not A.is_cuda
    if host:
        C_h = C
        if C_h is None:
            m_ = A.shape[0] if transa.upper() == "N" else A.shape[1]
            n_ = B.shape[1] if transb.upper() == "N" else B.shape[0]
            C_h = torch.empty((n_, m_), dtype=A.dtype, pin_memory=True).t()
        return _gemm_host(A, B, C_h, alpha, beta, transa, transb, variant, handle)
    dtype = A.dtype
    if dtype not in (torch.float64, torch.float32) or B.dtype != dtype:
        raise TypeError("A and B must both be float64 or both float32")
    esz = 8 if dtype == torch.float64 else 4
    ta, tb = transa.upper(), transb.upper()
    m = A.shape[0] if ta == "N" else A.shape[1]
    k = A.shape[1] if ta == "N" else A.shape[0]
    n = B.shape[1] if tb == "N" else B.shape[0]
    kb = B.shape[0] if tb == "N" else B.shape[1]
    if kb != k:
        raise ValueError(f"inner dimensions differ: op(A) is {m}x{k}, op(B) is {kb}x{n}")
    if C is None:
        if beta != 0.0:
            raise ValueError("C is required when beta != 0")
        C = torch.empty((n, m), dtype=dtype, device=A.device).t()
    if C.dtype != dtype or tuple(C.shape) != (m, n):
        raise ValueError(f"C must be {m}x{n} {dtype}")
    lda, ldb, ldc = _colmajor_ld(A, "A"), _colmajor_ld(B, "B"), _colmajor_ld(C, "C")
    h = handle or default_handle()
    h.bind_stream()
    h.ensure_workspace(ta, tb, m, n, k, esz)
    name = ENTRY[(variant, esz)]
    rc = _gemm_call(name, h.h, ta, tb, m, n, k, alpha, A.data_ptr(), lda, B.data_ptr(), ldb,
                    beta, C.data_ptr(), ldc)
    if rc != GFIP_OK:
        raise GemmError(rc, name)
    return C


def syrk(A, C=None, alpha: float = 1.0, beta: float = 0.0, uplo: str = "L", trans: str = "N",
         handle: Handle | None = None):
    """The triangle ``uplo`` of ``C := alpha*A*A^T + beta*C`` (trans 'N', A n x k) or
    ``alpha*A^T*A + beta*C`` (trans 'T', A k x n) on column-major CUDA tensors; the other
    triangle of C is left as it is (allocated, and left uninitialised, when C is None; beta
    must then be 0).  Asynchronous on torch's current stream.  Returns C."""
    import torch
    dtype = A.dtype
    if dtype not in (torch.float64, torch.float32):
        raise TypeError("A must be float64 or float32")
    esz = 8 if dtype == torch.float64 else 4
    tr, up = trans.upper(), uplo.upper()
    n = A.shape[0] if tr == "N" else A.shape[1]
    k = A.shape[1] if tr == "N" else A.shape[0]
    if C is None:
        if beta != 0.0:
            raise ValueError("C is required when beta != 0")
        C = torch.empty((n, n), dtype=dtype, device=A.device).t()
    if C.dtype != dtype or tuple(C.shape) != (n, n):
        raise ValueError(f"C must be {n}x{n} {dtype}")
    lda, ldc = _colmajor_ld(A, "A"), _colmajor_ld(C, "C")
    h = handle or default_handle()
    h.bind_stream()
    h.ensure_syrk_workspace(up, tr, n, k, esz)
    rc = gfip_syrk(esz, h.h, up, tr, n, k, alpha, A.data_ptr(), lda, beta, C.data_ptr(), ldc)
    if rc != GFIP_OK:
        raise GemmError(rc, "gfip_syrk")
    return C
