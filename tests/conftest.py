import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA GPU in this environment")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(autouse=True)
def _error_record_scope(request):
    """Attribute the relative errors the GPU parity tests compute to the
    running test (reported at the end of the session)."""
    try:
        import gpu_helpers
    except Exception:  # pragma: no cover
        yield
        return
    gpu_helpers.CURRENT["test"] = request.node.nodeid
    yield
    gpu_helpers.CURRENT["test"] = None


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """The largest relative Frobenius error each GPU parity test measured
    (FP32 results against the FP64 oracle fed the FP32-rounded inputs, FP64
    against the oracle), one line per test; with TG_PARITY_LOG set, the same
    as JSON in that file."""
    try:
        import gpu_helpers
    except Exception:  # pragma: no cover
        return
    worst = {}
    for test, err in gpu_helpers.ERRORS:
        if test is not None:
            worst[test] = max(worst.get(test, 0.0), err)
    if not worst:
        return
    terminalreporter.write_sep("-", "largest relative Frobenius error per parity test")
    for test in sorted(worst):
        terminalreporter.write_line(f"{worst[test]:.3e}  {test}")
    path = os.environ.get("TG_PARITY_LOG")
    if path:
        import json
        with open(path, "w") as fh:
            json.dump(worst, fh, indent=1, sort_keys=True)
