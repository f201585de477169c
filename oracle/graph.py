"""k-NN affinity graph and its symmetric normalisation (oracle, FP64).

Sec. 3: the n x n adjacency is sparse, symmetric, nonnegative and zero-diagonal;
it is normalised as W = D^-1/2 A D^-1/2 with D = diag(A 1).
Sec. 5.1: neighbours are the top k by dot product and the pairwise similarity is
(v^T z)_+^3.

Readings where the paper is silent:
* self is excluded from its own neighbour list; ties in similarity go to the
  smaller index;
* "union" keeps an edge if either endpoint lists the other (weight = the larger
  of the two directed weights); "mutual" keeps it only if both do (the smaller);
* edges whose weight is 0 (s <= 0) are not stored;
* a node of degree 0 gets D^-1/2 := 0, so its row and column of W are zero.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

CHUNK = 512


def knn_rows(X: np.ndarray, rows: np.ndarray, k: int) -> tuple[np.ndarray, np.ndarray]:
    """Top-k neighbours (by dot product, self excluded) of the given rows.

    Returns (idx, sim), both (len(rows), k), ordered by decreasing similarity
    with ties going to the smaller index.  FP64 throughout.  The k-th largest
    similarity of a row is found first; every entry at least that large is a
    candidate, and the candidates are ordered by (-s, index) exactly.
    """
    X = np.asarray(X, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    idx = np.empty((rows.size, k), dtype=np.int64)
    sim = np.empty((rows.size, k), dtype=np.float64)
    for s in range(0, rows.size, CHUNK):
        rr = rows[s:s + CHUNK]
        S = X[rr] @ X.T
        S[np.arange(rr.size), rr] = -np.inf          # no self loop
        kth = -np.partition(-S, k - 1, axis=1)[:, k - 1]
        for t in range(rr.size):
            cand = np.nonzero(S[t] >= kth[t])[0]
            order = cand[np.lexsort((cand, -S[t, cand]))][:k]   # decreasing s, then smaller id
            idx[s + t] = order
            sim[s + t] = S[t, order]
    return idx, sim


def directed_weights(X: np.ndarray, k: int, gamma: float = 3.0) -> sp.csr_matrix:
    """A_dir[i, j] = max(s_ij, 0)^gamma for j among the k neighbours of i."""
    n = X.shape[0]
    idx, sim = knn_rows(X, np.arange(n), k)
    w = np.maximum(sim, 0.0) ** gamma
    A = sp.csr_matrix((w.ravel(), (np.repeat(np.arange(n), k), idx.ravel())), shape=(n, n))
    A.eliminate_zeros()
    return A


def symmetrize(A_dir: sp.csr_matrix, sym: str = "union") -> sp.csr_matrix:
    """Undirected adjacency from directed k-NN weights."""
    At = A_dir.T.tocsr()
    if sym == "union":
        A = A_dir.maximum(At)
    elif sym == "mutual":
        both = (A_dir != 0).multiply(At != 0)
        A = A_dir.minimum(At).multiply(both)
    else:
        raise ValueError(sym)
    A = sp.csr_matrix(A, dtype=np.float64)
    A.eliminate_zeros()
    A.sort_indices()
    return A


def adjacency(X: np.ndarray, k: int, gamma: float = 3.0, sym: str = "union") -> sp.csr_matrix:
    """Sparse symmetric adjacency A of the k-NN graph of X (Sec. 3, Sec. 5.1)."""
    return symmetrize(directed_weights(X, k, gamma), sym)


def normalize(A: sp.csr_matrix) -> tuple[sp.csr_matrix, np.ndarray]:
    """W = D^-1/2 A D^-1/2 with D = diag(A 1) (Sec. 3).  Returns (W, d^-1/2)."""
    d = np.asarray(A.sum(axis=1)).ravel()
    dinv = np.zeros_like(d)
    nz = d > 0
    dinv[nz] = 1.0 / np.sqrt(d[nz])
    Dm = sp.diags(dinv)
    W = (Dm @ A @ Dm).tocsr()
    W.sort_indices()
    return W, dinv


def degrees(A: sp.csr_matrix) -> np.ndarray:
    return np.asarray(A.sum(axis=1)).ravel()
