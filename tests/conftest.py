import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(autouse=True)
def _bounds_check_word():
    """Under VOFP_CHECKED=1 (the bounds-checked library) every test that used the library must leave its index
    tests clean: the check word's count is read, and cleared, after each test."""
    yield
    mod = sys.modules.get("paper_1907_00890_gb300.vofp")
    if os.environ.get("VOFP_CHECKED") != "1" or mod is None:
        return
    st, w = mod.vofp_debug_check_word(reset=True)
    assert st == 1, "VOFP_CHECKED=1 but the plain library is loaded"
    assert w["count"] == 0, "out-of-range index tests in the bounds-checked library: %r" % (w,)
