"""Shared pytest configuration.

Markers:
  gpu  -- needs a CUDA device and the compiled libdg (run on a GB300 machine).
Everything else runs on the CPU in a few minutes.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU test")
