import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def load_kat():
    path = os.path.join(ROOT, "tests", "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = line.split()
        rows.append((int(v[0]), [int(x, 16) for x in v[1:5]], [int(x, 16) for x in v[5:7]],
                     [int(x, 16) for x in v[7:11]]))
    return rows
