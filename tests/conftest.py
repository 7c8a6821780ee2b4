import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")
    config.addinivalue_line("markers", "device_status_error: the test leaves a device-side error in a "
                                       "workspace on purpose (its status is not checked at teardown)")


@pytest.fixture(autouse=True)
def _workspace_status_clean(request):
    """For GPU tests: every batch workspace a test stages must end with a clean
    status word, so that a device-side bounds check that skipped an access (or
    a bounded loop that ran out) fails the test instead of passing silently."""
    if request.node.get_closest_marker("gpu") is None or request.node.get_closest_marker("device_status_error"):
        yield
        return
    import paper_2408_07625_gb300 as nqs
    made = []
    orig = nqs.Batch.__init__

    def init(self, *args, **kwargs):
        orig(self, *args, **kwargs)
        made.append(self)

    nqs.Batch.__init__ = init
    try:
        yield
    finally:
        nqs.Batch.__init__ = orig
    for b in made:
        b.status()   # raises NQSError with the device-side error
