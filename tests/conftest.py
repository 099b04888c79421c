import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture
def launch_override():
    """Set library launch-shape overrides (``api.set_launch_override``) for one test:
    ``launch_override(kchunk=7, adj_plain=1)``; every value is restored afterwards."""
    from paper_2211_15634_gb300 import api
    saved = {}

    def set_(**values):
        for name, v in values.items():
            old = api.set_launch_override(name, int(v))
            saved.setdefault(name, old)

    yield set_
    for name, v in saved.items():
        api.set_launch_override(name, v)
