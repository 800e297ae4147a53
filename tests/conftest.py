import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: long-running full-size case")


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def gpu_lib():
    """The product binding on a GPU machine; a missing extension is an error, not a skip."""
    if not cuda_available():
        pytest.skip("no CUDA device")
    import paper_1405_3454_gb300 as cp
    cp.load()  # raises if libcudapre.so is missing or does not load
    return cp
