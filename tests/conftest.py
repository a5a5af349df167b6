"""Shared pytest configuration.

Markers: ``gpu`` marks tests that need a CUDA device (the parity tests of the
CUDA path); everything else runs on CPU.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (parity tests of the CUDA path)")
    config.addinivalue_line("markers", "slow: longer oracle runs")


@pytest.fixture(scope="session")
def built_lib():
    """Build (or reuse) liblbm_gb300.so and return its path."""
    from paper_1303_4624_gb300 import build
    return build.build()


@pytest.fixture(scope="session")
def lbm(built_lib):
    """The ctypes binding module (requires a built library)."""
    from paper_1303_4624_gb300 import lbm as _lbm
    return _lbm


def golden_rows(name):
    path = os.path.join(ROOT, "tests", "golden", name)
    with open(path) as f:
        return [l.split() for l in f if l.strip() and not l.startswith("#")]
