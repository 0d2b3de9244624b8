import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running test, collected after the others")


def pytest_collection_modifyitems(config, items):
    # long-running tests after the others, so that a quick failure elsewhere
    # shows first; the test_zz_* files (single-purpose entry points) at the
    # very end, after the slow tests too
    items.sort(key=lambda it: (os.path.basename(str(it.fspath)).startswith("test_zz"),
                               it.get_closest_marker("slow") is not None))
