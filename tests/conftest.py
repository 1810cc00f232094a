import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(autouse=True)
def _no_index_violations(request):
    """With SC_LIBRARY=checked (the bounds-checked library) every GPU test must
    leave the kernels' index-violation count at zero."""
    yield
    if os.environ.get("SC_LIBRARY") != "checked" or "gpu" not in request.keywords:
        return
    import torch
    if not torch.cuda.is_available():
        return
    from paper_2205_15000_b300 import sc
    torch.cuda.synchronize()
    v, checked = sc.sc_debug_bounds(reset=True)
    assert checked, "SC_LIBRARY=checked loaded a library without index checks"
    assert v == 0, f"{v} index violations in the kernels"
