import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")


@pytest.fixture(scope="session")
def orc():
    import oracle
    return oracle.load()


@pytest.fixture(scope="session")
def cudalib():
    """The built CUDA library (built here when missing); GPU tests only."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_14821_gb300 import build, binding
    build.build()
    return binding


@pytest.fixture(scope="session")
def handle(cudalib):
    h = cudalib.bp_lb_create(150, 1 << 16)
    yield h
    cudalib.bp_lb_destroy(h)
