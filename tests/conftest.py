import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU statistics")


def read_golden(name):
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.fixture(params=["numpy", "cxx"])
def impl(request):
    """The FP64 reference under test: the numpy one (``oracle.sbs``) or the plain C++
    program behind the same interface (``oracle.cxx``); pins run on both."""
    if request.param == "cxx":
        from oracle import cxx
        cxx.load()
        return cxx
    from oracle import sbs
    return sbs
