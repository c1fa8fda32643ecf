import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device and the compiled library")


@pytest.fixture(scope="session")
def lib():
    """The compiled C-ABI library through its Python binding (GPU tests only)."""
    from paper_1606_00807_gb300 import binding
    return binding.load()
