import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def orc():
    from oracle import relcp_oracle as O

    O.lib()
    return O


@pytest.fixture(scope="session")
def relcp_gpu():
    """The CUDA library through its Python binding; builds it if needed.
    Fails (does not skip) when there is no GPU, so that a GPU run cannot pass
    on a silent fallback."""
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU test collected without a CUDA device")
    from paper_2506_14097_gb300 import relcp

    relcp.load()
    return relcp
