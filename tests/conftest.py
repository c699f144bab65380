import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libisg")
    config.addinivalue_line("markers", "slow: oracle runs of several seconds")


def read_golden(name):
    """Rows of a whitespace-separated golden file, comments dropped."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def read_golden_text(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return "".join(line.strip() for line in f if line.strip() and not line.startswith("#"))


@pytest.fixture(scope="session")
def gpu_available():
    import torch
    return torch.cuda.is_available()
