import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU-only test")


def read_golden(name):
    """Parse a tests/golden fixture: '#' lines are citations/comments,
    other lines are 'key = value' (floats) or 'key = v1, v2, ...'."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = (s.strip() for s in line.split("=", 1))
            parts = [float(v) for v in val.split(",")]
            out[key] = parts[0] if len(parts) == 1 else parts
    return out


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.load()
    return oracle
