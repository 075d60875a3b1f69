import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the compiled library")
    config.addinivalue_line("markers", "slow: long-running case")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Print the per-operator maxima of the value error measures the parity tests
    logged (tests/helpers.py: value_errors), and write them as JSON where
    FE_PARITY_REPORT names a file."""
    try:
        from helpers import PARITY_LOG
    except ImportError:
        return
    if not PARITY_LOG:
        return
    tr = terminalreporter
    tr.section("value errors against the oracle (max over cases)")
    tr.write_line(f"{'case [form]':56s} {'normwise':>9s} {'sum|c|':>9s} {'resolved':>9s} "
                  f"{'plain':>9s} {'#unres':>7s} {'#entries':>9s}")
    for k in sorted(PARITY_LOG):
        v = PARITY_LOG[k]
        tr.write_line(f"{k:56s} {v['norm']:9.2e} {v['comp']:9.2e} {v['comp_res']:9.2e} {v['plain']:9.2e} "
                      f"{v['n_unres']:7d} {v['n']:9d}")
    path = os.environ.get("FE_PARITY_REPORT")
    if path:
        import json
        with open(path, "w") as f:
            json.dump(PARITY_LOG, f, indent=1, sort_keys=True)
