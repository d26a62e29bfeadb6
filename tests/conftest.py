import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU-side oracle work")


def ensure_library():
    """Builds libdmk_stokes.so in-tree if it is missing (nvcc cross-compiles without a GPU)."""
    lib = os.path.join(ROOT, "paper_2509_21471_gb300", "libdmk_stokes.so")
    if not os.path.exists(lib):
        from paper_2509_21471_gb300 import build as _b
        _b.build()
    return lib


@pytest.fixture(scope="session")
def dmk_lib():
    ensure_library()
    from paper_2509_21471_gb300 import dmk
    return dmk
