import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: long CPU-only test")


# Files whose tests run after every other test, in this order: the
# allocation-free entry point's test comes last, so that a run stopping at the
# first failure has run everything else when it fails.
RUN_LAST = ("test_gpu_noalloc.py",)


def pytest_collection_modifyitems(session, config, items):
    def rank(item):
        name = os.path.basename(str(item.fspath))
        return RUN_LAST.index(name) + 1 if name in RUN_LAST else 0
    items.sort(key=rank)   # stable: the collection order is kept within each rank


@pytest.fixture(scope="session")
def cuda_ok():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return True
