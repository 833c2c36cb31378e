"""Shared pytest configuration: the ``gpu`` marker and repository import path."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built liblbm")
    config.addinivalue_line("markers", "slow: long CPU-side physics run (still part of the default suite)")
