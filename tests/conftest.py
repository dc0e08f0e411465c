import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def cpp_oracle():
    from oracle import cpp_oracle

    cpp_oracle.load()
    return cpp_oracle


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library through its C-ABI binding; fails loudly if absent."""
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU test collected without a CUDA device")
    from paper_2501_03245_gb300 import ecc

    ecc.load()
    return ecc
