"""Observation vectors y (oracle, FP64).

Sec. 3: y is a sparse n x 1 vector whose non-zeros sit at the nearest
neighbours of the query item in the dataset and hold the corresponding
similarities.  Sec. 5.1 uses the top few neighbours and (v^T z)_+^3 as the
similarity.  Reading: y_i = max(s_i, 0)^gamma over the top-k_y database items
by dot product (ties to the smaller id); entries equal to 0 are not stored.
"""
from __future__ import annotations

import numpy as np


def observe(Xdb: np.ndarray, Q: np.ndarray, k_y: int, gamma: float = 3.0):
    """Returns (y_ptr[B+1], y_idx, y_val) with one segment per query, ids ascending."""
    Xdb = np.asarray(Xdb, dtype=np.float64)
    Q = np.atleast_2d(np.asarray(Q, dtype=np.float64))
    n = Xdb.shape[0]
    ids = np.arange(n)
    ptr = [0]
    idx_all, val_all = [], []
    for q in Q:
        s = Xdb @ q
        order = np.lexsort((ids, -s))[:k_y]
        v = np.maximum(s[order], 0.0) ** gamma
        keep = v > 0
        sel = np.argsort(order[keep], kind="stable")
        idx_all.append(order[keep][sel])
        val_all.append(v[keep][sel])
        ptr.append(ptr[-1] + int(keep.sum()))
    return (np.asarray(ptr, dtype=np.int64),
            np.concatenate(idx_all).astype(np.int64) if idx_all else np.zeros(0, np.int64),
            np.concatenate(val_all) if val_all else np.zeros(0))


def observe_regional(Xdb: np.ndarray, Q: np.ndarray, regions: int, k_y: int, gamma: float = 3.0):
    """Regional queries (reading: one observation per query image): the
    image's `regions` consecutive rows of Q each contribute their own top-k_y
    (observe above); the lists are concatenated, so a database item found by
    several regions carries the sum of their values.  (y_ptr, y_idx, y_val)
    with one segment per image."""
    p, i, v = observe(Xdb, Q, k_y, gamma)
    nimg = (len(p) - 1) // regions
    ptr = np.asarray([p[j * regions] for j in range(nimg)] + [p[nimg * regions]], dtype=np.int64)
    return ptr, i, v


def dense(n: int, y_ptr, y_idx, y_val) -> np.ndarray:
    """Scatter the sparse columns into a dense n x B float64 array."""
    B = len(y_ptr) - 1
    Y = np.zeros((n, B))
    for j in range(B):
        s, e = y_ptr[j], y_ptr[j + 1]
        np.add.at(Y[:, j], np.asarray(y_idx[s:e], dtype=np.int64), y_val[s:e])
    return Y
