import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libsbm")
    config.addinivalue_line("markers", "slow: oracle cases that take more than a few seconds")


@pytest.fixture(scope="session")
def libsbm():
    """Builds (if stale) and loads libsbm.so; returns the binding module."""
    from paper_2506_12899_gb300 import build as B
    B.build()
    import paper_2506_12899_gb300 as S
    S.load_library()
    return S
