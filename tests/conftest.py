import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libttsn.so")


def pytest_collection_modifyitems(config, items):
    # keep GPU tests from running where there is no GPU only when explicitly deselected;
    # otherwise a GPU test without a GPU fails loudly instead of being skipped.
    pass
