import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")


@pytest.fixture(scope="session")
def cuda_ready():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1412_1945_gb300 as ocq

    ocq.load()  # raises when the CUDA library is missing: no silent fallback
    return ocq
