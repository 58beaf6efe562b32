import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and libpget.so")
    config.addinivalue_line("markers", "slow: long-running CPU check")


@pytest.fixture(scope="session")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def torch():
    import torch as _torch
    if not _torch.cuda.is_available():
        pytest.skip("CUDA device required")
    return _torch


@pytest.fixture(scope="session")
def P(torch):
    from paper_2604_26745_gb300 import build, pget
    build.build()
    pget.load()
    return pget


@pytest.fixture(scope="session")
def ctx(P):
    c = P.Context(0)
    yield c
    c.close()
