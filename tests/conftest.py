import os
import sys

# the oracle's many tiny LAPACK calls run faster without BLAS thread fan-out
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def fr3d_lib():
    """The compiled C-ABI library (built in-tree); tests that need it skip when it is absent on CPU."""
    from paper_1703_01216_gb300 import fr3d
    return fr3d.load()
