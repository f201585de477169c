"""Pins for oracle.truncated (Temporal†)."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import diffusion as D
from oracle import graph, truncated as T


def make_g80():
    X, _ = synth.database(41, 80, 12, 4, 30.0, 30.0)
    A = graph.adjacency(X, 7)
    return X, A


@pytest.fixture(scope="module")
def g80():
    return make_g80()


def test_full_shortlist_is_temporal(g80):
    # S = every node (any order): the truncated system is the whole graph
    X, A = g80
    W, _ = graph.normalize(A)
    y = np.zeros(80)
    y[[4, 9, 60]] = [1.0, 0.5, 0.2]
    S = np.random.default_rng(0).permutation(80)
    xs, _ = T.temporal_truncated(A, S, y, 0.9, 1e-13, 500)
    assert np.allclose(xs, D.closed_form(W, y, 0.9).ravel()[S], atol=1e-11)


def test_matches_dense_solve_built_by_loops(g80):
    # the renormalised subgraph rebuilt entry by entry from A, solved directly
    X, A = g80
    q = X[11] + 0.3 * X[50]
    S = T.shortlist(X, q, 30)
    Ad = A.toarray()
    s = len(S)
    sub = [[Ad[S[a], S[b]] for b in range(s)] for a in range(s)]
    deg = [sum(row) for row in sub]
    Ws = np.array([[sub[a][b] / np.sqrt(deg[a] * deg[b]) if deg[a] > 0 and deg[b] > 0 else 0.0 for b in range(s)]
                   for a in range(s)])
    y = np.zeros(80)
    y[S[:5]] = [1.0, 0.8, 0.6, 0.4, 0.2]
    y[S[-1]] += 0.1
    y[[i for i in range(80) if i not in set(S)][:3]] = 5.0  # outside S: dropped
    ys = y[S]
    want = (1 - 0.95) * np.linalg.solve(np.eye(s) - 0.95 * Ws, ys)
    got, _ = T.temporal_truncated(A, S, y, 0.95, 1e-13, 500)
    assert np.allclose(got, want, atol=1e-11)
    # invariants: x_S >= (1 - alpha) y_S, and per connected component of the
    # subgraph sqrt(d)^T x = sqrt(d)^T y (the eigenvalue-1 direction, h(1) = 1)
    assert np.all(got >= (1 - 0.95) * ys - 1e-12)
    Ws_sp, dinv = T.subsystem(A, S)
    ncomp, lab = sp.csgraph.connected_components(Ws_sp, directed=False)
    sd = np.where(dinv > 0, 1.0 / np.where(dinv > 0, dinv, 1.0), 0.0)
    for c in range(ncomp):
        m = lab == c
        assert sd[m] @ got[m] == pytest.approx(sd[m] @ ys[m], rel=1e-10, abs=1e-12)


def test_shortlist_order_and_ties():
    X = np.array([[1.0, 0.0], [0.0, 1.0], [1.0, 0.0], [0.6, 0.8], [-1.0, 0.0]])
    q = np.array([1.0, 0.0])
    got = T.shortlist(X, q, 4)
    brute = sorted(range(5), key=lambda i: (-float(X[i] @ q), i))[:4]
    assert list(got) == brute == [0, 2, 3, 1]
