import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running case")


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA extension, built in-tree; a GPU test fails loudly without it."""
    import torch

    if not torch.cuda.is_available():
        pytest.fail("gpu-marked test needs CUDA")
    from paper_2603_23343_gb300 import binding

    return binding
