import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def coeff_table():
    from paper_2007_06289_gb300 import iir_fit
    return iir_fit.load_table()


@pytest.fixture(scope="session")
def fbp():
    """The built library's Python binding (builds libfbp.so in-tree if it is stale)."""
    from paper_2007_06289_gb300 import binding, build
    build.build()
    binding.load_library()
    return binding
