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


@pytest.fixture(scope="session")
def cfg1_data():
    """The 2,000-node workload (d=128, 20 vMF components, k=30, 16 queries,
    top-10 observations), built entirely by the oracle in fp64."""
    import numpy as np
    import synth
    from oracle import graph, observe, spectral, diffusion
    c = synth.get_config("cfg1")
    X, lab = synth.database(c.seed, c.n, c.d, c.ncl, c.kappa_lo, c.kappa_hi, c.sizes)
    Qv = synth.queries(c.seed, c.batch, c.d, c.ncl, c.kappa_lo, c.kappa_hi, c.sizes)
    A = graph.adjacency(X, c.k, c.gamma)
    W, dinv = graph.normalize(A)
    yp, yi, yv = observe.observe(X, Qv, c.k_y, c.gamma)
    Y = observe.dense(c.n, yp, yi, yv)
    lam, U = spectral.eigh_desc(W)
    xstar = diffusion.closed_form(W, Y, c.alpha)
    return {"cfg": c, "X": X, "Q": Qv, "A": A, "W": W, "dinv": dinv, "yp": yp, "yi": yi, "yv": yv, "Y": Y,
            "lam": lam, "U": U, "xstar": xstar}


@pytest.fixture(scope="session")
def gpu_ctx():
    import paper_1807_08692_gb300 as hd
    ctx = hd.Context(0)
    yield ctx
    ctx.close()
