import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_collection_modifyitems(config, items):
    # GPU tests are skipped, not failed, where there is no GPU, so that a plain
    # `pytest tests/` on a CPU machine stays green; `-m gpu` selects them explicitly.
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA GPU on this machine")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_sessionfinish(session, exitstatus):
    # Under the bounds-checked library (L1LINE_LIB=.../libl1line_checks.so)
    # every GPU test ran with its kernel indices checked: no index may have
    # been out of range.
    lib = os.environ.get("L1LINE_LIB", "")
    if not lib.endswith("libl1line_checks.so"):
        return
    try:
        import torch
        if not torch.cuda.is_available():
            return
        from paper_2402_16712_gb300 import l1line
        hits, line = l1line.check_hits()
    except Exception as e:  # pragma: no cover
        print(f"\nbounds-checked build: counters unreadable ({e})")
        session.exitstatus = 1
        return
    print(f"\nbounds-checked build: {hits} out-of-range kernel indices"
          + (f" (the last at source line {line})" if hits else ""))
    if hits != 0:
        session.exitstatus = 1
