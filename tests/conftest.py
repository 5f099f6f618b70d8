import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: oracle runs that take tens of seconds")


def _cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _cuda_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device in this environment")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture
def product_algorithm(request):
    """Run a GPU test with the given exact-product algorithm, restoring AUTO after."""
    import paper_1810_01478_gb300 as hk
    hk.load()
    hk.hk_set_product_algorithm(request.param)
    yield request.param
    hk.hk_set_product_algorithm(hk.HK_PRODUCT_AUTO)
