"""Shared pytest configuration.

Markers:
  gpu -- needs a CUDA device (the parity tests proper); everything else runs on
         the CPU (oracle pins, host logic, C-ABI exports, multi-process gloo).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: test needs a CUDA GPU (GB300, sm_103a)")


def pytest_collection_modifyitems(config, items):
    # A gpu test that runs without a device must fail loudly, never fall back:
    # only skip when the run explicitly deselects gpu tests.
    pass


@pytest.fixture(scope="session")
def golden_dir():
    return os.path.join(ROOT, "tests", "golden")
