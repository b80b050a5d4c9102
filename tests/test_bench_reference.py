"""bench.py's reference arm (the oracle on the host cores) on CPU: one JSON line with the
keys of the bench contract, the GPU arm's metric and config for the same arguments, a
cpu_baseline that describes the run and an e2e object without copies."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--size", "96",
                          "--steps", "2", "--warmup", "3"], cwd=ROOT, capture_output=True,
                         text=True, timeout=600, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out
    r = json.loads(lines[0])
    assert r["impl"] == "reference"
    assert r["metric"] == "f64 gemm throughput (fused)"
    assert r["unit"] == "GFLOP/s" and r["higher_is_better"] is True
    assert r["value"] > 0 and r["ms_per_step"] > 0
    assert (r["n_gpus"], r["steps"], r["warmup"]) == (1, 2, 3)
    assert r["dtype"] == "f64" and r["data"] == "synthetic" and r["vs_baseline"] is None
    cfg = r["config"]
    assert (cfg["m"], cfg["n"], cfg["k"]) == (96, 96, 96)
    assert (cfg["lda"], cfg["ldb"], cfg["ldc"]) == (103, 103, 103)
    assert cfg["workload"].startswith("f64 gemm m=n=k=96 N/N lda=ldb=ldc=103")
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == r["value"] and cb["cores"] >= 1
    assert cb["sample"]
    assert r["e2e"] == {"value": r["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
