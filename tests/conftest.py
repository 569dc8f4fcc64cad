import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (run on a B300 box)")


@pytest.fixture(scope="session")
def cuda_lib():
    """The product library on a GPU; GPU tests fail loudly if it cannot be loaded."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_01203_b300 import binding
    return binding.lib()
