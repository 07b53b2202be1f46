import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def cuda():
    """The CUDA device for -m gpu tests; builds the library if it is stale."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_29291_gb300 import build as B
    B.build()
    return torch.device("cuda:0")


@pytest.fixture(scope="session")
def R(cuda):
    from paper_2605_29291_gb300 import rapdb
    return rapdb
