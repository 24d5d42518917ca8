"""Shared pytest configuration: the ``gpu`` marker and small fixtures."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def syn():
    from paper_2507_20802_gb300 import synthetic
    return synthetic


def load_golden(name):
    return dict(np.load(os.path.join(GOLDEN, name), allow_pickle=False))
