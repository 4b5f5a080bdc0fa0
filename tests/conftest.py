import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session", autouse=True)
def _built_library(request):
    """GPU sessions build the CUDA library once (no-op when up to date)."""
    if any(item.get_closest_marker("gpu") for item in request.session.items):
        from paper_2111_01083_gb300.build import build_library
        build_library()
