import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")


def golden_constants():
    out = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, val = line.split()[:2]
            out[name] = float(val)
    return out


def golden_velocities():
    rows = [list(map(int, l.split())) for l in open(os.path.join(GOLDEN, "d3q19_velocity_matrix.txt"))
            if l.strip() and not l.startswith("#")]
    return np.array(rows, dtype=np.int64).T  # (19, 3)


@pytest.fixture(scope="session")
def paper_e():
    return golden_velocities()


@pytest.fixture(scope="session")
def paper_const():
    return golden_constants()
