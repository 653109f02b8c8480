"""Shared pytest configuration.

Tests marked ``gpu`` need a CUDA device and the compiled CUDA library; everything else runs on
CPU (the oracle and its pins, the host-side logic, the C-ABI symbol checks, gloo process tests).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled CUDA library")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle
