import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def _cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _cuda_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture
def report(request):
    """Appends one JSON record per call to $HAP_REPORT_DIR/parity_report.jsonl
    (when that variable is set): the measured errors behind each assertion."""
    import json
    import time

    def _report(**values):
        d = os.environ.get("HAP_REPORT_DIR")
        if not d:
            return
        os.makedirs(d, exist_ok=True)
        rec = {"test": request.node.nodeid, "time": time.time(), **values}
        with open(os.path.join(d, "parity_report.jsonl"), "a") as f:
            f.write(json.dumps(rec, default=float) + "\n")

    return _report
