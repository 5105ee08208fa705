import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running case")
    if os.environ.get("TSDF_CHECKED") == "1":
        # the suite runs against the checked library (range checks on every
        # device index): make sure it is built
        from paper_2608_08287_gb300.build import build_library
        build_library(checked=True)
