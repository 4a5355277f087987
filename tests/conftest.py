import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libgh.so")


@pytest.fixture(scope="session")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="session")
def ctx(torch_cuda):
    """A libgh context on cuda:0; builds the library first (a failed build is
    an error, not a skip: there is no CPU fallback)."""
    from paper_2307_16550_gb300 import build, gh
    build.build()
    c = gh.Context(0)
    yield c
    c.close()
