import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_addoption(parser):
    parser.addoption("--run-large", action="store_true", default=False,
                     help="also run the full-size configurations (tests marked large)")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")
    config.addinivalue_line("markers", "large: a full-size configuration (tens to hundreds of GB, "
                                       "minutes); runs only with --run-large")


def pytest_collection_modifyitems(config, items):
    if config.getoption("--run-large"):
        return
    skip = pytest.mark.skip(reason="full-size configuration: run with --run-large")
    for item in items:
        if item.get_closest_marker("large") is not None:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle
