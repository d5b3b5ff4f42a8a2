import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU oracle case")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover
        return False


@pytest.fixture(scope="session")
def tlq():
    """The CUDA library's binding with one context on device 0 (GPU tests only)."""
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2112_10239_gb300 import binding
    ctx = binding.Context(device=0)
    yield ctx
    ctx.close()
