"""Shared pytest configuration.

Markers: ``gpu`` for tests that need a CUDA device (parity of the CUDA path
against the oracle); everything else runs on the CPU.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle


def build_flusi():
    """Build libflusi.so if needed, then import the binding."""
    import __graft_entry__
    __graft_entry__._build_module().build()
    import paper_1506_06513_gb300
    return paper_1506_06513_gb300
