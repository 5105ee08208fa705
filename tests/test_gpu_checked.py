"""The checked build on the GPU: every pool, table, coordinate and image index
range-checked before use (the stand-in for a memory checker, which is not
available here). Parity tests of every fusion strategy run in a child process
with TSDF_CHECKED=1, against the checked library: results must still equal
the oracle and no status may report BOUNDS (each test asserts OK statuses, and
an index out of range would set the BOUNDS bit and return TSDF_ERR_BOUNDS)."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SUBSET = ("room_640x480_every_mode or random_tiny_frames_split_walk or boundaries or "
          "pool_overflow or table_overflow or high_load_factor or layout_sums or "
          "empty_and_invalid or without_colour or caller_memory")


def test_parity_subset_under_range_checks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_08287_gb300.build import build_library
    build_library(checked=True)
    env = dict(os.environ, TSDF_CHECKED="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join("tests", "test_gpu_parity.py"), "-k", SUBSET],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and "failed" not in r.stdout, tail
