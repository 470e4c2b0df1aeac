import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def _gpu_ready() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def gpu():
    """The built CUDA library on cuda:0; GPU tests fail loudly if it is missing."""
    if not _gpu_ready():
        pytest.fail("GPU test collected without a CUDA device")
    import torch
    from paper_1806_09819_gb300 import build as B, leea
    B.build()
    leea.load_library()
    torch.cuda.set_device(0)
    return leea
