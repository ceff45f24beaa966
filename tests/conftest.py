import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled library")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def vga():
    """The CUDA library (built in-tree if stale).  GPU tests fail loudly when it cannot run."""
    from paper_2406_04177_gb300 import build

    build.build()
    import paper_2406_04177_gb300 as v

    v.load_library()
    return v
