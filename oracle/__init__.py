"""Plain FP64 GEMM oracle (CPU) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and reference
legs may import this package.  The product library (``paper_2302_08417_gb300``) never
imports it and shares no code with it.

The arithmetic lives in ``gemm_oracle.c`` (the GEMM of GEMMFIP Sec. 2.1, extended to the BLAS
dgemm semantics ``C := alpha*op(A)*op(B) + beta*C``); this module only compiles it with gcc
and marshals numpy buffers through ctypes.  Matrices are passed as flat float64 numpy arrays
holding column-major storage with a leading dimension, exactly as a BLAS caller would.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gemm_oracle.c")
_SRCS = [_SRC] + [os.path.join(_HERE, f) for f in ("syrk_oracle.c", "trmm_oracle.c",
                                                     "trsm_oracle.c")]
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle sources into oracle/_build/liboracle.so (gcc, no contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and all(os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-std=c99", "-Wall", "-shared", "-fPIC"] + _SRCS + ["-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, dbl, ptr = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
            lib.oracle_gemm.argtypes = [ctypes.c_char, ctypes.c_char, i64, i64, i64,
                                        dbl, ptr, i64, ptr, i64, dbl, ptr, i64, ctypes.c_int]
            lib.oracle_gemm.restype = ctypes.c_int
            lib.oracle_gemm_entries.argtypes = [ctypes.c_char, ctypes.c_char, i64, i64, i64,
                                                dbl, ptr, i64, ptr, i64, dbl, ptr, i64,
                                                i64, ptr, ptr, ptr, ctypes.c_int, ctypes.c_int]
            lib.oracle_gemm_entries.restype = ctypes.c_int
            lib.oracle_syrk.argtypes = [ctypes.c_char, ctypes.c_char, i64, i64, dbl, ptr,
                                        i64, dbl, ptr, i64]
            lib.oracle_syrk.restype = ctypes.c_int
            lib.oracle_trmm.argtypes = [ctypes.c_char, ctypes.c_char, ctypes.c_char,
                                        ctypes.c_char, i64, i64, dbl, ptr, i64, ptr, i64]
            lib.oracle_trmm.restype = ctypes.c_int
            lib.oracle_trsm.argtypes = lib.oracle_trmm.argtypes
            lib.oracle_trsm.restype = ctypes.c_int
            lib.oracle_max_threads.argtypes = []
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, name):
    if a is None:
        return None
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise TypeError(f"{name} must be a contiguous float64 numpy array")
    return a


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def gemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, nthreads=1) -> int:
    """In place ``C := alpha*op(A)*op(B) + beta*C`` on flat column-major float64 buffers.

    Returns the BLAS info code (0, or minus the position of the first bad argument)."""
    lib = _load()
    A = _f64(A, "A")
    B = _f64(B, "B")
    C = _f64(C, "C")
    return int(lib.oracle_gemm(transa.encode(), transb.encode(), m, n, k, float(alpha),
                               _ptr(A), lda, _ptr(B), ldb, float(beta), _ptr(C), ldc,
                               int(nthreads)))


def entries(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc, ii, jj,
            absval=False, nthreads=1) -> np.ndarray:
    """Entries ``(ii[t], jj[t])`` of ``alpha*op(A)*op(B) + beta*C0`` (same roundings as
    :func:`gemm`), or with ``absval`` the bound term ``|alpha||op(A)||op(B)| + |beta||C0|``."""
    lib = _load()
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    if ii.shape != jj.shape:
        raise ValueError("ii and jj must have the same shape")
    out = np.empty(ii.shape, dtype=np.float64)
    rc = lib.oracle_gemm_entries(transa.encode(), transb.encode(), m, n, k, float(alpha),
                                 _ptr(_f64(A, "A")), lda, _ptr(_f64(B, "B")), ldb,
                                 float(beta), _ptr(_f64(C0, "C0")), ldc, ii.size,
                                 _ptr(ii), _ptr(jj), _ptr(out), int(bool(absval)),
                                 int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_gemm_entries returned {rc}")
    return out


def gemm_result(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc,
                nthreads=1) -> np.ndarray:
    """Out-of-place convenience: returns a new flat buffer holding the updated C."""
    C = np.array(C0, dtype=np.float64, copy=True)
    rc = gemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, nthreads)
    if rc != 0:
        raise ValueError(f"oracle_gemm returned {rc}")
    return C


def abs_bound(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc,
              nthreads=1) -> np.ndarray:
    """``|alpha|*|op(A)|*|op(B)| + |beta|*|C0|`` for every entry, as an m x n array.

    This is the magnitude term of the elementwise error bound; every entry is formed by the
    same loop as :func:`entries` with ``absval``."""
    if m == 0 or n == 0:
        return np.zeros((m, n))
    ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    v = entries(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc,
                ii.ravel(), jj.ravel(), absval=True, nthreads=nthreads)
    return v.reshape(m, n)


def syrk(uplo, trans, n, k, alpha, A, lda, beta, C, ldc) -> int:
    """In place on C (flat float64, column-major, leading dimension ldc): the triangle uplo of
    alpha*A*A^T + beta*C (trans 'N', A n x k) or alpha*A^T*A + beta*C (trans 'T', A k x n).
    Returns 0 or minus the reference-BLAS position of the first bad argument."""
    lib = _load()
    return lib.oracle_syrk(uplo.encode(), trans.encode(), n, k, float(alpha),
                           _ptr(_f64(A, "A")), lda, float(beta), _ptr(_f64(C, "C")), ldc)


def syrk_result(uplo, trans, n, k, alpha, A, lda, beta, C0, ldc) -> np.ndarray:
    """Out-of-place convenience: returns a new flat buffer holding the updated C."""
    C = np.array(C0, dtype=np.float64, copy=True)
    rc = syrk(uplo, trans, n, k, alpha, A, lda, beta, C, ldc)
    if rc != 0:
        raise ValueError(f"oracle_syrk returned {rc}")
    return C


def trmm(side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb) -> int:
    """In place on B (flat float64, column-major): alpha*op(A)*B (side 'L') or alpha*B*op(A)
    (side 'R') with A triangular.  Returns 0 or minus the reference-BLAS position of the
    first bad argument."""
    lib = _load()
    return lib.oracle_trmm(side.encode(), uplo.encode(), transa.encode(), diag.encode(), m, n,
                           float(alpha), _ptr(_f64(A, "A")), lda, _ptr(_f64(B, "B")), ldb)


def trmm_result(side, uplo, transa, diag, m, n, alpha, A, lda, B0, ldb) -> np.ndarray:
    """Out-of-place convenience: returns a new flat buffer holding the updated B."""
    B = np.array(B0, dtype=np.float64, copy=True)
    rc = trmm(side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb)
    if rc != 0:
        raise ValueError(f"oracle_trmm returned {rc}")
    return B


def trsm(side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb) -> int:
    """In place on B (flat float64, column-major): X with op(A) X = alpha B (side 'L') or
    X op(A) = alpha B (side 'R'), A triangular.  Returns 0 or minus the reference-BLAS
    position of the first bad argument."""
    lib = _load()
    return lib.oracle_trsm(side.encode(), uplo.encode(), transa.encode(), diag.encode(), m, n,
                           float(alpha), _ptr(_f64(A, "A")), lda, _ptr(_f64(B, "B")), ldb)


def trsm_result(side, uplo, transa, diag, m, n, alpha, A, lda, B0, ldb) -> np.ndarray:
    """Out-of-place convenience: returns a new flat buffer holding the solution X."""
    B = np.array(B0, dtype=np.float64, copy=True)
    rc = trsm(side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb)
    if rc != 0:
        raise ValueError(f"oracle_trsm returned {rc}")
    return B
