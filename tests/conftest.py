import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def libpath():
    """The built liblbm.so (built here if missing; loading needs no GPU)."""
    from paper_1710_07073_gb300 import build, lbm
    if not os.path.exists(lbm.LIB_PATH):
        build.build()
    return lbm.LIB_PATH
