"""Seeded synthetic GEMM operands in BLAS column-major storage.

This module only draws numbers and lays them out; it holds none of the GEMM arithmetic, so
both the CUDA path and the CPU oracle can be fed from it.

A column-major ``rows x cols`` matrix with leading dimension ``ld >= rows`` is stored as a
flat buffer of ``ld * cols`` elements; element ``(r, c)`` sits at ``r + c*ld``.  The gap rows
``rows .. ld-1`` of every column are filled with a sentinel (NaN by default): a kernel that
reads them, or writes them in C, is caught by the NaN or by the changed sentinel.

Distributions (the workloads of GEMM performance sweeps: i.i.d. uniform[-1, 1]; small
integers for bit-exact checks; log-uniform magnitudes with random sign for scaling
stress):
  * ``"uniform"``: i.i.d. U[-1, 1].
  * ``"int"``: i.i.d. integers in [-lim, lim] (default 4), exact in FP32 and FP64.
  * ``"logmag"``: magnitude 10**U[-4, 4], random sign.
"""
from __future__ import annotations

from dataclasses import dataclass
import math

import numpy as np

SENTINEL = np.nan


def _draw(rng: np.random.Generator, size: int, dist: str, int_lim: int) -> np.ndarray:
    if dist == "uniform":
        return rng.uniform(-1.0, 1.0, size)
    if dist == "int":
        return rng.integers(-int_lim, int_lim + 1, size).astype(np.float64)
    if dist == "logmag":
        mag = 10.0 ** rng.uniform(-4.0, 4.0, size)
        sign = np.where(rng.integers(0, 2, size) == 0, -1.0, 1.0)
        return mag * sign
    raise ValueError(f"unknown distribution {dist!r}")


def colmajor(rng: np.random.Generator, rows: int, cols: int, ld: int, dtype=np.float64,
             dist: str = "uniform", int_lim: int = 4, sentinel=SENTINEL) -> np.ndarray:
    """Flat column-major buffer of ``max(ld*cols, 1)`` elements, gap rows = sentinel."""
    if ld < max(1, rows):
        raise ValueError("ld must be >= max(1, rows)")
    buf = np.full((max(cols, 0), ld), sentinel, dtype=np.float64)
    if rows > 0 and cols > 0:
        vals = _draw(rng, rows * cols, dist, int_lim).reshape(cols, rows)
        buf[:, :rows] = vals
    flat = buf.reshape(-1)
    if flat.size == 0:
        flat = np.full(1, sentinel, dtype=np.float64)
    return flat.astype(dtype)


def as_matrix(flat: np.ndarray, rows: int, cols: int, ld: int) -> np.ndarray:
    """View of the ``rows x cols`` logical matrix held in a flat column-major buffer."""
    if rows == 0 or cols == 0:
        return np.zeros((rows, cols), dtype=flat.dtype)
    return flat[: ld * cols].reshape(cols, ld)[:, :rows].T


def is_notrans(t: str) -> bool:
    return t in ("N", "n")


@dataclass
class Problem:
    transa: str
    transb: str
    m: int
    n: int
    k: int
    alpha: float
    beta: float
    A: np.ndarray
    lda: int
    B: np.ndarray
    ldb: int
    C0: np.ndarray
    ldc: int

    @property
    def dtype(self):
        return self.A.dtype

    @property
    def rows_a(self) -> int:
        return self.m if is_notrans(self.transa) else self.k

    @property
    def cols_a(self) -> int:
        return self.k if is_notrans(self.transa) else self.m

    @property
    def rows_b(self) -> int:
        return self.k if is_notrans(self.transb) else self.n

    @property
    def cols_b(self) -> int:
        return self.n if is_notrans(self.transb) else self.k


def problem(seed: int, transa: str = "N", transb: str = "N", m: int = 64, n: int = 64,
            k: int = 64, alpha: float = 1.0, beta: float = 0.5, pad_a: int = 0,
            pad_b: int = 0, pad_c: int = 0, dtype=np.float64, dist: str = "uniform",
            int_lim: int = 4, c_sentinel=SENTINEL) -> Problem:
    """One seeded GEMM problem.  ``lda = rows(A) + pad_a`` (rows(A) = m for 'N', k for
    'T'), likewise ``ldb = rows(B) + pad_b`` and ``ldc = m + pad_c``; every ld is at least 1.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    rows_a = m if is_notrans(transa) else k
    cols_a = k if is_notrans(transa) else m
    rows_b = k if is_notrans(transb) else n
    cols_b = n if is_notrans(transb) else k
    lda = max(1, rows_a + pad_a)
    ldb = max(1, rows_b + pad_b)
    ldc = max(1, m + pad_c)
    A = colmajor(rng, rows_a, cols_a, lda, dtype, dist, int_lim)
    B = colmajor(rng, rows_b, cols_b, ldb, dtype, dist, int_lim)
    C0 = colmajor(rng, m, n, ldc, dtype, dist, int_lim, sentinel=c_sentinel)
    return Problem(transa, transb, m, n, k, float(alpha), float(beta), A, lda, B, ldb, C0, ldc)


def unit_roundoff(dtype) -> float:
    """u = 2**-53 for float64, 2**-24 for float32."""
    return 2.0 ** -53 if np.dtype(dtype) == np.float64 else 2.0 ** -24


def config_sizes() -> list[int]:
    """The square sizes of the GEMM size sweep, 16 .. 16384: 16, then 2**j (j = 5..14) and
    3*2**(j-1) (j = 5..13), i.e. 16, 32, 48, 64, 96, ..., 8192, 12288, 16384 (20 sizes)."""
    sizes = {16}
    sizes.update(2 ** j for j in range(5, 15))
    sizes.update(3 * 2 ** (j - 1) for j in range(5, 14))
    return sorted(sizes)


def sample_indices(rng: np.random.Generator, m: int, n: int, count: int, full_rows: int = 0,
                   full_cols: int = 0):
    """Sampled (i, j) result positions: ``count`` random entries plus whole rows/columns."""
    ii = [rng.integers(0, m, count)] if count else []
    jj = [rng.integers(0, n, count)] if count else []
    for r in rng.choice(m, size=min(full_rows, m), replace=False) if full_rows else []:
        ii.append(np.full(n, r))
        jj.append(np.arange(n))
    for c in rng.choice(n, size=min(full_cols, n), replace=False) if full_cols else []:
        ii.append(np.arange(m))
        jj.append(np.full(m, c))
    if not ii:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(ii).astype(np.int64), np.concatenate(jj).astype(np.int64)


def log2_ceil(x: int) -> int:
    return 0 if x <= 1 else math.ceil(math.log2(x))
