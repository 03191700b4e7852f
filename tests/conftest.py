import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def read_golden(name):
    """Parse a tests/golden fixture: '## section' headers followed by rows of numbers."""
    path = os.path.join(ROOT, "tests", "golden", name)
    sections = {}
    cur = None
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("# "):
                continue
            if line.startswith("## "):
                cur = line[3:].strip()
                sections[cur] = []
                continue
            sections[cur].append([float(t) for t in line.split()])
    return {k: np.array(v if len(v) > 1 else v[0]) for k, v in sections.items()}


def pytest_sessionstart(session):
    # The native library is built in-tree; compile it if it is missing or stale
    # (nvcc cross-compiles without a GPU).
    from paper_1008_1700_gb300.build import build
    build()
