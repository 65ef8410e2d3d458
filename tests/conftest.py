import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# the oracle's node loops may use the host's cores (results do not depend on
# the thread count); a run can pin it with ORACLE_THREADS
try:
    _cores = len(os.sched_getaffinity(0))
except AttributeError:  # pragma: no cover
    _cores = os.cpu_count() or 1
os.environ.setdefault("ORACLE_THREADS", str(max(1, min(_cores, 32))))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU run of the oracle")


def pytest_collection_modifyitems(config, items):
    """Skip GPU tests cleanly when no GPU is present; they are selected with -m gpu."""
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)
