import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (run on the GB300 box)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def cfg1():
    from paper_2110_11644_gb300 import synth
    return synth.config_pocket(1), synth.config_ligands(1), synth.config_params(1)


@pytest.fixture(scope="session")
def cfg2_pocket():
    from paper_2110_11644_gb300 import synth
    return synth.config_pocket(2)
