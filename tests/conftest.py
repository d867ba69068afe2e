import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libscan.so")
    config.addinivalue_line("markers", "slow: long CPU check, runs only with SCAN_SLOW_TESTS=1")


def pytest_collection_modifyitems(config, items):
    if os.environ.get("SCAN_SLOW_TESTS") == "1":
        return
    skip = pytest.mark.skip(reason="slow; set SCAN_SLOW_TESTS=1")
    for item in items:
        if "slow" in item.keywords:
            item.add_marker(skip)


def load_golden(name):
    """Parse a tests/golden/*.txt fixture into a dict of fields."""
    path = os.path.join(ROOT, "tests", "golden", name)
    out = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            out.setdefault(key, []).append(rest)
    return out
