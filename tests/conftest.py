import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libeat")


@pytest.fixture(scope="session")
def large_tt():
    """The 200,000-stop network (about 46 M connections), generated once per session."""
    import synth
    return synth.large()


@pytest.fixture(scope="session")
def large_sc(large_tt):
    """The large network's connections sorted for the oracle (Algorithm 1), once."""
    import oracle
    return oracle.SortedConnections(large_tt)
