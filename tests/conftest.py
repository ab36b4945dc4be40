import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")
    # (registered here too, for a run without the pytest-timeout plugin,
    # where the mark is then inert)
    config.addinivalue_line("markers", "timeout(seconds): fail a test that runs longer")
