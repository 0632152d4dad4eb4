import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libmgq")
    config.addinivalue_line("markers", "slow: long statistical test")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    oracle.lib()
    return oracle


@pytest.fixture(scope="session")
def mgqlib():
    """The built libmgq (compiled in-tree if missing or stale)."""
    from paper_1510_04675_gb300 import _lib, build

    build.build()
    return _lib.load()


@pytest.fixture(scope="session")
def gpu(mgqlib):
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1510_04675_gb300 import api

    return api
