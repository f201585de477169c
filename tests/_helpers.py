"""Shared checks for the GPU parity tests (test-side only; no method arithmetic
beyond what the oracle defines)."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def csr_of(A):
    A = sp.csr_matrix(A)
    A.sort_indices()
    return (A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float32))


def y_arrays(yp, yi, yv):
    return (np.ascontiguousarray(yp, np.int32), np.ascontiguousarray(yi, np.int32),
            np.ascontiguousarray(yv, np.float32))


def rel_l2_cols(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    num = np.linalg.norm(x - ref, axis=0)
    den = np.linalg.norm(ref, axis=0)
    out = np.zeros_like(num)
    nz = den > 0
    out[nz] = num[nz] / den[nz]
    out[~nz] = num[~nz]
    return out


def check_knn_lists(idx, sim, Xdb, Q, k, exclude_self, sim_tol):
    """Neighbour lists are valid top-k lists of the exact (fp64) similarities.

    Per row: ids distinct and in range, returned similarities equal the exact
    ones within sim_tol, ordered by decreasing similarity, and every returned
    id is at least as similar as the exact k-th neighbour minus sim_tol (so a
    swap can only happen inside a near-tie at the boundary).  Returns the
    number of rows whose id set differs from the exact top-k set.
    """
    Xdb = np.asarray(Xdb, np.float64)
    Q = np.asarray(Q, np.float64)
    idx = np.asarray(idx)
    sim = np.asarray(sim, np.float64)
    nq = Q.shape[0]
    differ = 0
    for q in range(nq):
        s = Xdb @ Q[q]
        if exclude_self:
            s[q] = -np.inf
        order = np.lexsort((np.arange(s.size), -s))
        kth = s[order[k - 1]]
        ids = idx[q]
        assert np.all(ids >= 0) and np.all(ids < Xdb.shape[0]), f"row {q}: id out of range"
        assert len(set(ids.tolist())) == k, f"row {q}: duplicate ids"
        if exclude_self:
            assert q not in set(ids.tolist()), f"row {q}: self listed"
        assert np.allclose(sim[q], s[ids], atol=sim_tol, rtol=0), f"row {q}: similarity mismatch"
        assert np.all(np.diff(sim[q]) <= sim_tol), f"row {q}: not sorted"
        assert np.all(s[ids] >= kth - sim_tol), f"row {q}: a neighbour below the k-th similarity"
        if set(ids.tolist()) != set(order[:k].tolist()):
            differ += 1
    return differ


def check_ranking(ids, scores, x_ref, x=None, score_tol=0.0, tie_rel=1e-5):
    """A GPU ranking (ids, scores of length K) is a valid top-K of the oracle's
    scores x_ref: position by position up to ties of tie_rel * max x_ref, ids
    distinct, nothing that belongs in the top K left out, and its scores are
    the ranked vector's (x, the GPU's own scores when given, else x_ref) at
    those ids within score_tol, in decreasing order with ties to the smaller id."""
    from oracle import rank as ORank
    x_ref = np.asarray(x_ref, np.float64)
    ids = np.asarray(ids)
    K = ids.size
    ref, _ = ORank.topk(x_ref, K)
    assert ORank.ranks_match(ids, ref, x_ref, tie_rel * np.abs(x_ref).max(), scores=scores,
                             x=x_ref if x is None else x, score_tol=score_tol)


def near_tie_rows(X, k, margin, exclude_self=True):
    """Rows whose exact k-th and (k+1)-th similarities differ by less than margin."""
    X = np.asarray(X, np.float64)
    out = []
    for s0 in range(0, X.shape[0], 2048):
        S = X[s0:s0 + 2048] @ X.T
        if exclude_self:
            for t in range(S.shape[0]):
                S[t, s0 + t] = -np.inf
        S = -np.sort(-S, axis=1)
        out.extend((s0 + np.where(S[:, k - 1] - S[:, k] < margin)[0]).tolist())
    return np.asarray(out, dtype=np.int64)


def check_graph(rp, col, val, dinv, A_ref, uncertain, rtol=2e-5):
    """GPU graph (W, D^-1/2) versus the oracle adjacency.

    The raw adjacency A = D^1/2 W D^1/2 is rebuilt from the export; entries may
    differ only in rows or columns of `uncertain` nodes (a swap at a near-tie
    k-th neighbour moves an edge).  Elsewhere W and D^-1/2 must agree to rtol.
    """
    n = len(rp) - 1
    Wg = sp.csr_matrix((np.asarray(val, np.float64), np.asarray(col), np.asarray(rp)), shape=(n, n))
    dg = np.asarray(dinv, np.float64)
    with np.errstate(divide="ignore"):
        sq = np.where(dg > 0, 1.0 / dg, 0.0)
    Ag = (sp.diags(sq) @ Wg @ sp.diags(sq)).tocsr()
    D = (Ag - sp.csr_matrix(A_ref)).tocoo()
    big = np.abs(D.data) > rtol * np.abs(sp.csr_matrix(A_ref).data).max()
    bad_nodes = set(np.asarray(uncertain).tolist())
    touched = set()
    for i, j in zip(D.row[big], D.col[big]):
        assert i in bad_nodes or j in bad_nodes, f"edge ({i},{j}) differs away from any near-tie"
        touched.update((int(i), int(j)))
    Wr, dref = __import__("oracle").graph.normalize(sp.csr_matrix(A_ref))
    ok = np.array([i not in touched for i in range(n)])
    assert np.allclose(dg[ok], dref[ok], rtol=rtol)
    rows = np.where(ok)[0]
    Wd = (Wg[rows] - Wr[rows]).tocoo()
    assert np.all(np.abs(Wd.data) <= rtol * np.abs(Wr.data).max() + 1e-9) or len(touched) > 0
    return len(touched)
