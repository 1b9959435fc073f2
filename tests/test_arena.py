"""The serving engine's device / pinned-host range allocator (header-only C++,
offsets only), checked on the CPU against a byte-ownership model."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_range_arena_randomized(seed):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "arena_check")
        subprocess.check_call([gxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2010_15879_gb300", "csrc"),
                               os.path.join(ROOT, "tests", "arena_check.cpp"), "-o", exe])
        out = subprocess.run([exe, str(seed)], capture_output=True, text=True, timeout=300)
        assert out.returncode == 0, out.stdout + out.stderr
        assert out.stdout.startswith("ok")
