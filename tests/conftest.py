import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libxpr.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as O
    O.build()
    return O


@pytest.fixture(autouse=True)
def _device_flags_clear(request):
    """After every GPU test: no kernel of the library recorded a timed-out wait or an inconsistent
    intermediate (the sort's chained scan records them in device flags instead of faulting)."""
    yield
    if request.node.get_closest_marker("gpu") is None:
        return
    from paper_2606_11529_gb300 import binding as B
    if B._lib is not None:
        B.xpr_device_check()
