"""Pins for oracle.graph and oracle.observe: pure-Python brute force and invariants."""
import numpy as np
import pytest

import synth
from oracle import graph, observe


def _py_knn(X, k):
    """Neighbour lists by explicit loops: sort (-s, j) over j != i."""
    n = len(X)
    lists = []
    for i in range(n):
        cand = []
        for j in range(n):
            if j == i:
                continue
            s = sum(float(X[i][t]) * float(X[j][t]) for t in range(len(X[i])))
            cand.append((-s, j))
        cand.sort()
        lists.append([(j, -ms) for ms, j in cand[:k]])
    return lists


@pytest.mark.parametrize("sym", ["union", "mutual"])
def test_adjacency_matches_loops(sym):
    X, _ = synth.database(3, 25, 6, 3, 20.0, 20.0)
    k, gamma = 4, 3.0
    lists = _py_knn(X, k)
    want = {}
    directed = {}
    for i, lst in enumerate(lists):
        for j, s in lst:
            directed[(i, j)] = max(s, 0.0) ** gamma
    for (i, j), w in directed.items():
        back = directed.get((j, i))
        if sym == "union":
            v = w if back is None else max(w, back)
        else:
            if back is None:
                continue
            v = min(w, back)
        if v > 0:
            want[(i, j)] = v
            want[(j, i)] = v
    A = graph.adjacency(X, k, gamma, sym).tocoo()
    got = {(int(i), int(j)): float(v) for i, j, v in zip(A.row, A.col, A.data)}
    assert set(got) == set(want)
    for key in want:
        assert got[key] == pytest.approx(want[key], rel=1e-12)


def test_graph_invariants(small_graph):
    A, W, dinv = small_graph["A"], small_graph["W"], small_graph["dinv"]
    Ad = A.toarray()
    assert np.allclose(Ad, Ad.T)
    assert np.all(np.diag(Ad) == 0)
    assert np.all(Ad >= 0)
    d = Ad.sum(1)
    sd = np.sqrt(d)
    # W D^1/2 1 = D^-1/2 A 1 = D^1/2 1: sqrt(d) is an eigenvector with eigenvalue 1.
    assert np.allclose(W @ sd, sd, rtol=1e-12, atol=1e-14)
    assert np.allclose(dinv, 1 / np.sqrt(d))


def test_degree_zero_node():
    # A node that nobody lists mutually has no edge; its D^-1/2 is 0 by the reading.
    X = np.array([[1, 0], [0.99, 0.141], [0.98, 0.199], [-1, 0.0]], dtype=np.float64)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    A = graph.adjacency(X, 1, 3.0, "mutual")
    W, dinv = graph.normalize(A)
    iso = np.where(np.asarray(A.sum(1)).ravel() == 0)[0]
    assert iso.size >= 1
    assert np.all(dinv[iso] == 0)
    assert np.all(W.toarray()[iso] == 0)


def test_knn_rows_tie_rule():
    # Rows 1, 2 and 3 are identical: row 0 sees three equal similarities.
    X = np.array([[1, 0], [0, 1], [0, 1], [0, 1], [-1, 0]], dtype=np.float64)
    X[0] = [0.6, 0.8]
    idx, sim = graph.knn_rows(X, np.array([0]), 2)
    assert list(idx[0]) == [1, 2]


def test_observe_matches_loops():
    X, _ = synth.database(5, 40, 5, 3, 10.0, 10.0)
    Q = synth.queries(5, 3, 5, 3, 10.0, 10.0)
    ptr, idx, val = observe.observe(X, Q, 6, 3.0)
    for j, q in enumerate(Q):
        s = [(-sum(float(q[t]) * float(X[i][t]) for t in range(5)), i) for i in range(40)]
        s.sort()
        want = sorted((i, max(-ms, 0.0) ** 3) for ms, i in s[:6] if -ms > 0)
        got = list(zip(idx[ptr[j]:ptr[j + 1]], val[ptr[j]:ptr[j + 1]]))
        assert [g[0] for g in got] == [w[0] for w in want]
        assert np.allclose([g[1] for g in got], [w[1] for w in want], rtol=1e-12)


def test_observe_dense_scatter():
    ptr = np.array([0, 2, 3])
    Y = observe.dense(5, ptr, np.array([1, 4, 0]), np.array([0.5, 0.25, 2.0]))
    assert Y.shape == (5, 2)
    assert Y[1, 0] == 0.5 and Y[4, 0] == 0.25 and Y[0, 1] == 2.0 and Y.sum() == 2.75


def test_observe_regional_is_the_sum_of_region_observations():
    # reading for regional queries: an image's observation vector is the sum of
    # its regions' observation vectors (computed one region at a time here)
    X, _ = synth.database(6, 50, 5, 3, 10.0, 10.0)
    Q = synth.queries(6, 3 * 4, 5, 3, 10.0, 10.0)
    ptr, idx, val = observe.observe_regional(X, Q, 4, 5, 3.0)
    Y = observe.dense(50, ptr, idx, val)
    assert Y.shape == (50, 3)
    for img in range(3):
        want = np.zeros(50)
        for reg in range(4):
            p1, i1, v1 = observe.observe(X, Q[img * 4 + reg], 5, 3.0)
            want += observe.dense(50, p1, i1, v1)[:, 0]
        assert np.allclose(Y[:, img], want, rtol=0, atol=0)
