import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libadg.so")
    config.addinivalue_line("markers", "slow: long-running CPU check")
    # used by pytest-timeout where installed; registered here so that it is known without it
    config.addinivalue_line("markers", "timeout(seconds): limit on a test's run time")
