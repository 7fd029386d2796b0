import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libgi.so")
    config.addinivalue_line("markers", "slow: long-running parity case")


def pytest_collection_modifyitems(config, items):
    # GPU tests are skipped (not failed) when no GPU is visible so that a
    # plain `pytest` on a CPU host still runs the oracle pins.
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA GPU visible")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    # Shares of gradient elements that needed the FP32 conditioning clause
    # (tests/tolerances.py), the largest per test group, beside the share of
    # elements ill-conditioned enough to use it.
    try:
        from tolerances import CLAUSE_LOG, CLAUSE_SHARE_MAX
    except ImportError:
        return
    if not CLAUSE_LOG:
        return
    worst = {}
    for test, group, used, ill, n in CLAUSE_LOG:
        key = f"{test} {group}"
        if key not in worst or used > worst[key][0]:
            worst[key] = (used, ill, n)
    tr = terminalreporter
    tr.write_line(f"conditioning clause: largest share used per check (limit {CLAUSE_SHARE_MAX:.0%}), "
                  "beside the share with kappa above the threshold")
    for key, (used, ill, n) in sorted(worst.items(), key=lambda kv: -kv[1][0])[:12]:
        tr.write_line(f"  {used:8.4%} of {n:>7} (ill-conditioned {ill:7.4%})  {key}")
