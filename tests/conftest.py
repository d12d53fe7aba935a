import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def read_golden(name):
    """Rows of whitespace-separated tokens from tests/golden/<name>, comments skipped."""
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.fixture(scope="session")
def golden():
    return read_golden


@pytest.fixture(scope="session")
def mck():
    """The CUDA binding with libmck.so built for this machine (GPU tests only)."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_08159_gb300 import build

    build.build()
    import paper_1702_08159_gb300 as m

    torch.cuda.set_device(0)
    return m


@pytest.fixture(scope="session")
def dev():
    import torch

    return torch.device("cuda", 0)
