import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs on the GB300 box)")
    config.addinivalue_line("markers", "slow: full-size case (minutes of CPU oracle time)")


@pytest.fixture(scope="session")
def fxlib():
    """The built library (built here if missing; nvcc cross-compiles without a GPU)."""
    import paper_2604_22242_gb300 as fx
    from paper_2604_22242_gb300 import build as fxbuild
    fxbuild.build()
    fx.lib()
    return fx
