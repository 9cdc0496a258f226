import os
import sys

# one hardware work queue per stream for the concurrent serving lanes (set before CUDA starts)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import pytest  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built library")
    config.addinivalue_line("markers", "slow: oracle cases that take more than a few seconds")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def lib():
    """The CUDA library through its C-ABI binding (built in-tree by __graft_entry__.build)."""
    from paper_2310_16829_gb300 import lma
    return lma.load()


@pytest.fixture(scope="session", autouse=True)
def _built_library():
    """Every test runs against the in-tree library: build it once if this checkout has none."""
    from paper_2310_16829_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
