"""Ranking by decreasing score (oracle).

Sec. 3: items are ranked by decreasing order of the elements of x.
Reading: equal scores are ordered by the smaller (original) item id first.
Optional pooling: per-image score = sum of the scores of its consecutive
`seg` rows (regional descriptors, one image per segment).
"""
from __future__ import annotations

import numpy as np


def topk(x: np.ndarray, K: int) -> tuple[np.ndarray, np.ndarray]:
    """Top-K ids and scores of a score vector, decreasing, ties to the smaller id."""
    x = np.asarray(x)
    order = np.lexsort((np.arange(x.size), -x))[:K]
    return order.astype(np.int64), x[order]


def pooled(x: np.ndarray, seg: int) -> np.ndarray:
    """Per-image sum of `seg` consecutive rows."""
    x = np.asarray(x, dtype=np.float64)
    return x.reshape(-1, seg, *x.shape[1:]).sum(axis=1)


def ranks_match(ids_a, ids_b, score_ref: np.ndarray, tie: float) -> bool:
    """True when two rankings agree position by position up to score ties.

    At each position the ids must be equal or have reference scores within
    `tie` of each other.  Used by tests to compare a computed ranking with the
    oracle's when several orders are correct.
    """
    ids_a = np.asarray(ids_a)
    ids_b = np.asarray(ids_b)
    if ids_a.shape != ids_b.shape:
        return False
    for a, b in zip(ids_a, ids_b):
        if a != b and abs(score_ref[a] - score_ref[b]) > tie:
            return False
    return True
