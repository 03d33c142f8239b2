import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running oracle checks")


@pytest.fixture(scope="session")
def small_ground_state():
    """Oracle SCF ground state of the two-well system (24^3, N = 16)."""
    from paper_2410_09189_gb300 import inputs
    from oracle import groundstate
    s = inputs.small()
    gs = groundstate.ground_state(s, tol=1e-10)
    return s, gs
