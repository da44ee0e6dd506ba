import os
import sys

import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


def read_golden(name):
    """Rows of a whitespace table in tests/golden/<name>, comments dropped."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


@pytest.fixture(scope="session")
def golden():
    return read_golden


@pytest.fixture(scope="session")
def ppeel_lib():
    """libppeel.so, built in place if missing or stale (nvcc cross-compiles)."""
    from paper_1302_7014_b300 import _lib
    from paper_1302_7014_b300.build import build
    build()
    return _lib.load()


def cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
