import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libsense.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_finish(session):
    # The precision study's FP64 references take minutes: start them as soon as
    # the selected tests are known, so that they run beside the other GPU tests.
    if any("test_gpu_precision320" in item.nodeid for item in session.items):
        from tests import precision_refs

        precision_refs.start()
