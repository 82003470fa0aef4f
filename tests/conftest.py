import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a B300 (sm_103a) GPU")
    config.addinivalue_line("markers", "injects_wait_timeouts: the test makes bounded waits expire on purpose")


@pytest.fixture(autouse=True)
def no_expired_waits(request):
    """After every GPU test (except the one that injects them): no bounded
    wait of a tensor-core kernel expired, so no output was left incomplete."""
    yield
    if request.node.get_closest_marker("gpu") is None or request.node.get_closest_marker("injects_wait_timeouts"):
        return
    from paper_1904_08555_b300 import cj
    try:
        st = cj.stats()
    except cj.CJError as e:
        if e.status == cj.CJ_ERR_NOT_INITIALIZED:
            return
        raise
    assert st["wait_timeouts"] == 0, f"{st['wait_timeouts']} bounded waits expired"


def read_golden(name):
    """Parse a tests/golden/*.txt fixture: '#' comments, 'KEY v1 v2 ...' lines."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *vals = line.split()
            out[k] = vals
    return out
