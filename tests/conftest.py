"""Shared test set-up: the ``gpu`` marker and import paths.

Tests marked ``gpu`` need a CUDA device (a GB300); everything else runs on a
CPU-only machine.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")


GOLDEN = os.path.join(ROOT, "tests", "golden")


def load_golden(name):
    import numpy as np
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle
