"""Test configuration: the ``gpu`` marker and import paths.

``-m "not gpu"`` runs on any machine (oracle pins, host logic, ABI symbols);
``-m gpu`` needs a CUDA device and the built library.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device and the built gf2x library")
    config.addinivalue_line("markers", "slow: longer CPU test")
