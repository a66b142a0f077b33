import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def oracle_threads() -> int:
    return max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="session")
def nthreads():
    return oracle_threads()


def pytest_collection_modifyitems(config, items):
    """Tests marked slow (minutes of oracle time each) run only with DUGKS_SLOW=1."""
    if os.environ.get("DUGKS_SLOW") == "1":
        return
    skip = pytest.mark.skip(reason="slow oracle run; set DUGKS_SLOW=1")
    for item in items:
        if "slow" in item.keywords:
            item.add_marker(skip)
