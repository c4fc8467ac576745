import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU check")


@pytest.fixture(scope="session")
def oracle_lib():
    from oracle import oracle as orc

    return orc.load()


@pytest.fixture(scope="session")
def libpt():
    """Build (if stale) and load the CUDA library; nvcc cross-compiles without a GPU."""
    from paper_1004_0023_gb300 import build, pt

    build.build()
    return pt.load()


def has_gpu():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False
