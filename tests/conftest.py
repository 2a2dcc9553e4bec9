import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libcc.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def cclib():
    """Built libcc.so on a CUDA machine (GPU tests only)."""
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_1407_7105_gb300 import build, cc

    build.build()
    return cc


_IC_CACHE = {}


@pytest.fixture(scope="session")
def plummer_ic():
    """Cached seeded Plummer spheres: plummer_ic(n, seed) -> (m, x3, v3)."""
    from paper_1407_7105_gb300 import ics

    def get(n, seed=1):
        key = ("plummer", n, seed)
        if key not in _IC_CACHE:
            _IC_CACHE[key] = ics.plummer(n, seed=seed)
        return _IC_CACHE[key]

    return get
