"""The host thread pool that copies pageable rasters into the pinned ring
(step a2): compiled with g++ against its header and stress-tested on the CPU,
no GPU involved."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2104_14667_gb300", "csrc")


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_every_piece_runs_once_on_every_pool_width(tmp_path):
    exe = tmp_path / "copy_pool_stress"
    subprocess.run(["g++", "-std=c++17", "-O2", "-pthread", "-x", "c++", "-I", CSRC,
                    os.path.join(ROOT, "tests", "copy_pool_stress.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "failures 0" in out.stdout
