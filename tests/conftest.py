import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libfde")
    config.addinivalue_line("markers", "slow: oracle pins that take tens of seconds")


@pytest.fixture(scope="session")
def golden():
    import json
    with open(os.path.join(ROOT, "tests", "golden", "paper_tables.json")) as f:
        return json.load(f)


@pytest.fixture(scope="session")
def gpu():
    """The built library and torch on cuda:0; skips when no GPU is visible."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1912_13304_gb300 as fde
    from paper_1912_13304_gb300 import build
    build.build()
    fde.lib()
    return torch
