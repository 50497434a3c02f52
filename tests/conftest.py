import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def fdl():
    """The CUDA binding, with libfdl.so built for this machine (GPU tests only)."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1901_06919_gb300 import build as B

    B.build()
    import paper_1901_06919_gb300 as F

    F.load()
    return F
