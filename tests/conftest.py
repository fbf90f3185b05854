import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300) and the built library")


def golden(name):
    """Rows of a whitespace-separated golden fixture, comments dropped."""
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def paper_constant(name):
    for row in golden("paper_constants.txt"):
        if row[0] == name:
            return float(row[1])
    raise KeyError(name)
