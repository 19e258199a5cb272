import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: full-size cases (minutes)")


def pytest_collection_modifyitems(config, items):
    """GPU tests fail loudly (never skip silently) when no GPU is present and
    they were selected; on a CPU-only host the default -m "not gpu" run
    deselects them."""
    return
