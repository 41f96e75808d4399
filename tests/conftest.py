import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_sessionstart(session):
    """Compile liblider.so first if it is missing (a fresh checkout): the
    tests load the library, and building it needs only nvcc, no GPU."""
    lib = os.path.join(ROOT, "paper_2205_00970_b300", "liblider.so")
    if not os.path.exists(lib):
        from paper_2205_00970_b300 import build_lib
        build_lib.build()
