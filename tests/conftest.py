import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


@pytest.fixture(scope="session")
def lib():
    """The built C-ABI library through its ctypes binding (built on demand)."""
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1707_05058_gb300 import cdsdp
    return cdsdp
