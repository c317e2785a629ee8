import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")
    config.addinivalue_line("markers", "run_last: GPU tests of a newly added path; collected after the "
                                       "others so that a failure under -x does not hide them")


def pytest_collection_modifyitems(session, config, items):
    items.sort(key=lambda it: it.get_closest_marker("run_last") is not None)
