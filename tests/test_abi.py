"""The C-ABI library without a GPU: it loads, exports every symbol include/gemmfip.h
declares, and reports reference-BLAS argument codes before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2302_08417_gb300 import build as libbuild
from paper_2302_08417_gb300 import gemmfip as g

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gemmfip.h")


@pytest.fixture(scope="module")
def lib():
    libbuild.build(probe=False)
    return g.load()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gfip_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_expected_entry_points():
    syms = declared_symbols()
    for name in ("gfip_dgemm", "gfip_sgemm", "gfip_dgemm_direct", "gfip_sgemm_direct",
                 "gfip_dgemm_pack_then_compute", "gfip_sgemm_pack_then_compute",
                 "gfip_create", "gfip_destroy", "gfip_set_stream", "gfip_set_workspace",
                 "gfip_workspace_size", "gfip_get_status"):
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert name in g.SIGNATURES, f"binding lacks {name}"


def test_test_hooks_stay_out_of_the_public_header(lib):
    """The failure-path hook of the emulation is declared in the library's internal testing
    header only, and the library still exports it for the GPU test."""
    text = open(HEADER).read()
    assert "gfip_debug" not in text
    testing = open(os.path.join(ROOT, "paper_2302_08417_gb300", "csrc", "gfip_testing.h")).read()
    assert "gfip_debug_ozaki_timeout(" in testing
    assert hasattr(lib, "gfip_debug_ozaki_timeout")


def test_error_strings(lib):
    assert g.error_string(0) == "success"
    assert "transa" in g.error_string(-1)
    assert "workspace" in g.error_string(g.GFIP_ERR_WORKSPACE)
    assert "capturing" in g.error_string(g.GFIP_ERR_CAPTURE)


ARGS = dict(transa="N", transb="N", m=2, n=2, k=2, alpha=1.0, A=16, lda=2, B=16, ldb=2,
            beta=0.0, C=16, ldc=2)
BAD = [
    (dict(transa="X"), -1), (dict(transb="q"), -2), (dict(m=-1), -3), (dict(n=-1), -4),
    (dict(k=-1), -5), (dict(m=3, ldc=3), -8), (dict(transa="T", k=3, ldb=3), -8),
    (dict(k=3, lda=2), -10), (dict(transb="T", n=3, ldc=2, lda=2), -10),
    (dict(m=3, lda=3), -13), (dict(m=0, n=0, k=0, lda=0), -8),
]


@pytest.mark.parametrize("entry", sorted(g.ENTRY.values()))
@pytest.mark.parametrize("change,code", BAD)
def test_blas_argument_codes_without_device(lib, entry, change, code):
    a = dict(ARGS)
    a.update(change)
    rc = g._gemm_call(entry, 0, a["transa"], a["transb"], a["m"], a["n"], a["k"], a["alpha"],
                      a["A"], a["lda"], a["B"], a["ldb"], a["beta"], a["C"], a["ldc"])
    assert rc == code


def test_valid_arguments_with_null_handle_report_handle_error(lib):
    for entry in g.ENTRY.values():
        rc = g._gemm_call(entry, 0, "N", "N", 2, 2, 2, 1.0, 16, 2, 16, 2, 0.0, 16, 2)
        assert rc == g.GFIP_ERR_HANDLE
    assert g.gfip_set_stream(0, 0) == g.GFIP_ERR_HANDLE
    assert g.gfip_set_workspace(0, 0, 0) == g.GFIP_ERR_HANDLE
    assert g.gfip_workspace_size(0, "N", "N", 4, 4, 4, 8) == 0


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.gfip_create(ctypes.byref(h))
    assert rc in (g.GFIP_ERR_CUDA, g.GFIP_ERR_DEVICE)
    assert not h.value


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2302_08417_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "gemm_oracle" not in text, f
