"""The benchmark's output contract, checked on the CPU: the reference arm
(the oracle timed on the host, the only arm that runs without a GPU) prints
exactly one JSON line with the keys the contract names, and the kernel-source
hashes that gate the profiled DRAM traffic match the committed ncu summaries.
No GPU is needed."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--ref-n", "256"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in out, key
    assert out["impl"] == "reference" and out["value"] > 0 and out["higher_is_better"] is True
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] >= 1
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["d2h_bytes_per_step"] == 0
    assert out["e2e"]["value"] == out["value"]


def test_profiled_traffic_is_reported_only_for_matching_sources():
    # a committed ncu summary carries the hash of the kernel sources it was
    # taken on; the benchmark reports its DRAM traffic while they match and
    # null once the kernel has changed
    import re
    sys.path.insert(0, ROOT)
    import bench
    for prof, files, key in (("k_factor_dag_fp64.md", bench.QR_SOURCES, "16384x16384/nb128/ib16"),
                             ("k_lu_dag_fp64.md", bench.LU_SOURCES, "16384x16384/nb128/ib16"),
                             ("k_chol_dag_fp64.md", bench.CHOL_SOURCES, "16384x16384/nb128")):
        txt = open(os.path.join(ROOT, "profiles", prof)).read()
        match = re.search(r"source_hash:\s*([0-9a-f]+)", txt).group(1) == bench.kernel_source_hash(files)
        t = bench.profiled_traffic(key, prof, files)
        assert (t is not None and t > 0) == match
