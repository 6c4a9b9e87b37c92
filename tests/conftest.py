import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA path through the C ABI)")
    config.addinivalue_line("markers", "slow: longer CPU case")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def qlib():
    """The CUDA library, built in-tree if it is missing or stale (nvcc cross-compiles without a GPU)."""
    from paper_2011_04130_gb300 import _build

    _build.build()
    import paper_2011_04130_gb300 as q

    q.load_library()
    return q


@pytest.fixture(scope="session")
def gpu(qlib):
    """A library context on cuda:0 (GPU tests only)."""
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    ctx = qlib.Context(0)
    yield ctx
    torch.cuda.synchronize()
    ctx.close()
