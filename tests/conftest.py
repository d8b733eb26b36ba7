import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    oracle.lib()
    return oracle


@pytest.fixture(scope="session")
def g():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2512_19750_gb300 as lib

    return lib


@pytest.fixture(scope="session")
def gctx(g):
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    ctx = g.gace_create(0)
    yield ctx
    g.gace_destroy(ctx)


@pytest.fixture(scope="session")
def cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch.device("cuda:0")
