import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running test, collected after the others")


def pytest_collection_modifyitems(config, items):
    # long-running tests last, so that a quick failure elsewhere shows first
    items.sort(key=lambda it: it.get_closest_marker("slow") is not None)
