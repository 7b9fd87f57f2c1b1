import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU-only oracle runs")


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover
        return False


def _slow_selected(config):
    expr = (config.option.markexpr or "").replace(" ", "")
    return "slow" in expr and "notslow" not in expr


def pytest_collection_modifyitems(config, items):
    # slow CPU runs (tens of minutes of the FP64 oracle) only when asked for by
    # name (-m slow), so that the default CPU suite stays at a few minutes
    if not _slow_selected(config):
        skip_slow = pytest.mark.skip(reason="slow oracle run: select it with -m slow")
        for item in items:
            if "slow" in item.keywords:
                item.add_marker(skip_slow)
    if gpu_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device in this process")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)
