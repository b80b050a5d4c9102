"""Helpers for the GPU tests: run a seeded problem through the C ABI and compare with the
oracle.  Imported only by tests marked ``gpu``."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2302_08417_gb300 import gemmfip as g
from paper_2302_08417_gb300 import inputs

VARIANTS = ("fused", "direct", "pack_then_compute")
GUARD = 64  # sentinel elements after the end of C


class Runner:
    """One handle with a growing workspace; copies problems to the device and back."""

    def __init__(self):
        torch.cuda.set_device(0)
        self.dev = torch.device("cuda", 0)
        self.h = g.Handle()
        self.h.bind_stream()

    def run(self, p: inputs.Problem, variant="fused", policy=g.GFIP_PACK_AUTO, C_init=None,
            A_dev=None, B_dev=None, expect_rc=0, packer=g.GFIP_PACKER_AUTO):
        """Returns (C as a flat numpy buffer without the guard, guard, A after, B after)."""
        esz = p.A.dtype.itemsize
        A = A_dev if A_dev is not None else torch.from_numpy(p.A).to(self.dev)
        B = B_dev if B_dev is not None else torch.from_numpy(p.B).to(self.dev)
        c0 = p.C0 if C_init is None else C_init
        Cbuf = np.concatenate([c0, np.full(GUARD, np.nan, dtype=c0.dtype)])
        C = torch.from_numpy(Cbuf).to(self.dev)
        self.h.set_pack_policy(policy)
        self.h.set_packer(packer)
        self.h.ensure_workspace(p.transa, p.transb, p.m, p.n, p.k, esz)
        name = g.ENTRY[(variant, esz)]
        rc = g._gemm_call(name, self.h.h, p.transa, p.transb, p.m, p.n, p.k, p.alpha,
                          A.data_ptr(), p.lda, B.data_ptr(), p.ldb, p.beta, C.data_ptr(), p.ldc)
        assert rc == expect_rc, f"{name} returned {rc} ({g.error_string(rc)})"
        torch.cuda.synchronize()
        out = C.cpu().numpy()
        self.h.set_pack_policy(g.GFIP_PACK_AUTO)
        self.h.set_packer(g.GFIP_PACKER_AUTO)
        return out[: c0.size], out[c0.size:]


def reference(p: inputs.Problem):
    """Oracle result (flat float64 buffer) and the bound term |alpha||A||B| + |beta||C0|."""
    A, B, C0 = (x.astype(np.float64) for x in (p.A, p.B, p.C0))
    ref = oracle.gemm_result(p.transa, p.transb, p.m, p.n, p.k, p.alpha, A, p.lda, B, p.ldb,
                             p.beta, C0, p.ldc, nthreads=4)
    ab = oracle.abs_bound(p.transa, p.transb, p.m, p.n, p.k, p.alpha, A, p.lda, B, p.ldb,
                          p.beta, C0, p.ldc, nthreads=4)
    return ref, ab


def tolerance(p: inputs.Problem, absterm):
    """2 * max(k, 2) * u * (|alpha||op(A)||op(B)| + |beta||C0|), u of the result type."""
    u = inputs.unit_roundoff(p.A.dtype)
    return 2.0 * max(p.k, 2) * u * absterm


def assert_close(p: inputs.Problem, got_flat, ref_flat=None, absterm=None, label=""):
    if ref_flat is None:
        ref_flat, absterm = reference(p)
    got = inputs.as_matrix(got_flat.astype(np.float64), p.m, p.n, p.ldc)
    ref = inputs.as_matrix(ref_flat, p.m, p.n, p.ldc)
    tol = tolerance(p, absterm)
    err = np.abs(got - ref)
    bad = ~(err <= tol)
    if bad.any():
        i, j = np.argwhere(bad)[0]
        raise AssertionError(
            f"{label} {p.transa}{p.transb} m={p.m} n={p.n} k={p.k} ld=({p.lda},{p.ldb},{p.ldc})"
            f" beta={p.beta}: {bad.sum()} entries out of bound; first ({i},{j}) got {got[i, j]!r}"
            f" want {ref[i, j]!r} tol {tol[i, j]:.3e}")


def assert_gap_untouched(p: inputs.Problem, got_flat, guard, C_init=None):
    """Rows m..ldc-1 of C and the guard after C keep their sentinels."""
    c0 = p.C0 if C_init is None else C_init
    if p.n > 0 and p.ldc > p.m:
        gap_got = got_flat.reshape(p.n, p.ldc)[:, p.m:]
        gap_0 = c0.reshape(p.n, p.ldc)[:, p.m:]
        assert np.array_equal(gap_got.view(np.uint8), gap_0.view(np.uint8)), "C gap rows written"
    assert np.all(np.isnan(guard)), "guard after C written"
