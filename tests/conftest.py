import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def small_graph():
    """A 60-node union k-NN graph from a 4-component vMF mixture (oracle-built)."""
    import numpy as np
    import synth
    from oracle import graph
    X, lab = synth.database(11, 60, 8, 4, 30.0, 30.0)
    A = graph.adjacency(X, 6)
    W, dinv = graph.normalize(A)
    return {"X": X, "A": A, "W": W, "dinv": dinv, "lab": lab, "n": 60}
