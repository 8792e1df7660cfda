import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session", autouse=True)
def checked_build_reports_no_violation():
    """With ZM_LIB=checked the whole suite runs on the checked build (libzm_checked.so, whose
    kernels count out-of-range indices instead of accessing them); at the end of the session
    the count must be zero."""
    yield
    if os.environ.get("ZM_LIB") != "checked":
        return
    from paper_2406_05490_gb300 import zm
    if zm._lib is None:  # no test loaded the library
        return
    hits, first, line = zm.zm_bounds_status(clear=True)
    assert zm.zm_checked_build() and hits == 0, \
        f"checked build: {hits} index violations, first index {first} at source line {line}"
