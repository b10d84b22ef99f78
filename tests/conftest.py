import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")


@pytest.fixture(scope="session")
def qtlib():
    """The built shared library (builds it in-tree if needed)."""
    from paper_2106_15740_gb300 import _build, binding
    _build.build()
    return binding.lib()
