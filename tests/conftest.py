import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# The oracle is dense small-matrix numpy; many BLAS threads only slow it down.
os.environ.setdefault("OMP_NUM_THREADS", "1")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device and the built libdpgmg.so")
    config.addinivalue_line("markers", "slow: oracle runs that take more than a few seconds")
