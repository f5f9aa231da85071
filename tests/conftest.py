import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: long-running case")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def rambo_lib():
    """The CUDA library, built for sm_103a and loaded (GPU tests only)."""
    if not gpu_available():
        pytest.fail("GPU test collected on a machine without a CUDA device")
    from paper_1910_04358_gb300 import rambo
    return rambo
