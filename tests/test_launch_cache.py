"""The library's per-device launch set-up memo (csrc/launch_cache.h), tested
on the host: compiled with g++ together with a fake set-up function and run
from several threads (no GPU, no CUDA call)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_launch_cache_once_per_device_and_kernel(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = tmp_path / "launch_cache_test"
    src = os.path.join(ROOT, "tests", "cpp", "launch_cache_test.cpp")
    inc = os.path.join(ROOT, "paper_0709_1272_gb300", "csrc")
    subprocess.run([gxx, "-std=c++17", "-O1", "-pthread", "-I", inc, src, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("OK")
