import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs on the GB300 box)")
    config.addinivalue_line("markers", "slow: long-running (full-size workloads)")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def mrsim():
    """The CUDA library binding; on a GPU machine a missing extension is an error."""
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2508_03960_gb300 import mrsim as m
    return m
