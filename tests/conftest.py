import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and libsk.so built for sm_103a")
    config.addinivalue_line("markers", "slow: long-running")


@pytest.fixture(scope="session")
def sk():
    """The CUDA binding with its library built in tree (fails loudly if the build fails)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_20195_gb300 import _build
    _build.build()
    from paper_2606_20195_gb300 import sk as skmod
    skmod.load()
    return skmod


@pytest.fixture(scope="session")
def dev():
    import torch
    return torch.device("cuda:0")
