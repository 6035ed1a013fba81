import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: long-running CPU oracle case")


def pytest_collection_modifyitems(config, items):
    try:
        import torch

        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(autouse=True)
def _device_waits_completed(request):
    """After every GPU test: no bounded device-side wait gave up (fhe_sync reports FHE_ETIMEOUT)."""
    yield
    if "gpu" not in request.keywords:
        return
    import paper_2607_05920_gb300 as fhe

    rc = fhe.lib.fhe_sync(None)
    assert rc == 0, f"fhe_sync after the test returned {rc}: {fhe.lib.fhe_last_error().decode()}"
