import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running")
    # a sanitizer run (tests/test_host_sanitize.py) loads another build of the library
    path = os.environ.get("COBS_TEST_LIBRARY")
    if path:
        from paper_1905_09624_gb300 import cobs
        cobs.lib(path=path)


def pytest_collection_modifyitems(config, items):
    # A GPU test on a machine without a GPU is skipped, never silently routed elsewhere.
    has_gpu = False
    if not os.environ.get("COBS_TEST_LIBRARY"):  # sanitizer runs are host-only
        try:
            import torch
            has_gpu = torch.cuda.is_available()
        except Exception:
            has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)
