import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built liblbm.so")
    config.addinivalue_line("markers", "slow: long CPU run")


def golden_path(name):
    return os.path.join(ROOT, "tests", "golden", name)


def read_matrix(name):
    """Read a printed matrix fixture into a list of Fractions rows."""
    from fractions import Fraction

    rows = []
    with open(golden_path(name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([Fraction(tok) for tok in line.split()])
    return rows


def read_values(name):
    out = {}
    with open(golden_path(name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()[:2]
            out[k] = float(v)
    return out
