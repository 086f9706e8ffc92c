"""Shared pytest set-up: the `gpu` marker and session fixtures.

Tests marked ``gpu`` need a CUDA device and the compiled sm_103a library;
everything else runs on the CPU (oracle pins, host logic, library symbols).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled CUDA library")
    config.addinivalue_line("markers", "slow: long CPU runs of the oracle")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle
