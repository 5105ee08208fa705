"""The range checks of the checked build (the stand-in for a memory checker)
exercised on the host: tests/check_bounds.cpp, compiled with and without
TSDF_CHECKED against csrc/tsdf_check.h, feeds them in-range and out-of-range
indices. No GPU: the checked kernels themselves run in the GPU suite with
TSDF_CHECKED=1."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "check_bounds.cpp")


@pytest.mark.parametrize("checked", [True, False])
def test_range_checks_on_the_host(tmp_path, checked):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path / ("check_on" if checked else "check_off"))
    cmd = [gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_2608_08287_gb300", "csrc"), SRC, "-o", exe]
    if checked:
        cmd.insert(1, "-DTSDF_CHECKED")
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout
