import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def gpu():
    """Build (if needed) and load the CUDA library; require a CUDA device."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_03972_gb300 import binding, build

    build.build()
    binding.load()
    return binding
