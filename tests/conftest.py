import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")


def read_golden(name):
    """Parse a tests/golden/*.txt case file: 'case NAME' ... 'end' blocks of key/values."""
    cases, cur = {}, None
    with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "case":
                cur = {}
                cases[parts[1]] = cur
            elif parts[0] == "end":
                cur = None
            else:
                vals = [float(v) for v in parts[1:]]
                cur[parts[0]] = vals if len(vals) > 1 or parts[0] in (
                    "t_offsets", "y", "dy", "expect_bins") else vals[0]
    return cases


@pytest.fixture(scope="session")
def golden_cases():
    return read_golden("hand_cases.txt")
