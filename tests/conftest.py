import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU case")


@pytest.fixture(scope="session")
def h2o8():
    """(H2O)8-like: 32 orbitals, L = 6.21 A, 48^3 grid, seed 1000."""
    from paper_2208_06097_gb300 import synth
    return synth.make_config("h2o8_48")


@pytest.fixture(scope="session")
def h2o8_oracle(h2o8):
    from oracle import oracle as O
    return O.apply_vxx(h2o8.phi, h2o8.cell, O.Params())


@pytest.fixture
def rng():
    return np.random.default_rng(12345)
