import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libfrlap extension")


@pytest.fixture(scope="session")
def frlap():
    """The product binding, loaded once per session (GPU tests only)."""
    import paper_1804_02718_gb300 as pkg
    return pkg
