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
def gpu_lib():
    """The CUDA library, built for sm_103a; fails loudly if it is missing."""
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a -m gpu test ran without a CUDA device")
    import paper_2004_06278_gb300 as sq

    sq.load()
    return sq
