import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_terminal_summary(terminalreporter):
    """Report how many mixed-path cases retained other ranks than the oracle
    (each then compared against the oracle truncated at the GPU's ranks)."""
    try:
        from _util import RANK_WINDOW_HITS
    except ImportError:
        return
    terminalreporter.write_line(f"mixed-path rank-window cases: {len(RANK_WINDOW_HITS)}")
    for line in RANK_WINDOW_HITS:
        terminalreporter.write_line(f"  {line}")
