import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")
    # temporary files of the tests (tmp_path) stay inside the tree, in an ignored folder
    if not config.option.basetemp:
        os.makedirs(os.path.join(ROOT, "tests", "_build"), exist_ok=True)
        config.option.basetemp = os.path.join(ROOT, "tests", "_build", "pytest_tmp")
