import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def metro():
    """The metro-shaped workload (~550k edges, 3.2M trips), generated once per
    test session (a module may override the name with its own fixture)."""
    from paper_2007_03614_b300 import synth
    net = synth.metro_network()
    return net, synth.metro_trips(net)
