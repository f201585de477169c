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


def ranks_match(ids, ids_ref, score_ref: np.ndarray, tie: float, scores=None, x=None,
                score_tol: float = 0.0) -> bool:
    """True when `ids` is a valid top-K ranking of `score_ref` up to score ties.

    `ids_ref` is the reference ranking (`topk(score_ref, K)`).  Required:
      * the same length as `ids_ref`, every id in [0, len(score_ref)), no id twice;
      * position by position, the ids are equal or their reference scores lie
        within `tie` of each other;
      * no item left out of `ids` has a reference score above the K-th
        reference score by more than `tie` (nothing that belongs in the top K
        is missing).
    With `scores` (the ranking's own scores) and `x` (the score vector it was
    ranked from) also required:
      * scores[p] equals x[ids[p]] within score_tol * max |x[ids]| (0: exactly);
      * the scores are non-increasing, and equal scores list the smaller id first
        (Sec. 3: decreasing order; ties to the smaller id).
    """
    ids = np.asarray(ids).astype(np.int64).ravel()
    ids_ref = np.asarray(ids_ref).astype(np.int64).ravel()
    score_ref = np.asarray(score_ref, dtype=np.float64).ravel()
    n = score_ref.size
    if ids.shape != ids_ref.shape:
        return False
    K = ids.size
    if K == 0:
        return True
    if ids.min() < 0 or ids.max() >= n:
        return False
    if np.unique(ids).size != K:
        return False
    differ = (ids != ids_ref) & (np.abs(score_ref[ids] - score_ref[ids_ref]) > tie)
    if np.any(differ):
        return False
    left_out = np.ones(n, dtype=bool)
    left_out[ids] = False
    if left_out.any() and score_ref[left_out].max() > score_ref[ids_ref[-1]] + tie:
        return False
    if scores is not None:
        sc = np.asarray(scores, dtype=np.float64).ravel()
        if sc.shape != ids.shape:
            return False
        xs = np.asarray(x, dtype=np.float64).ravel()[ids]
        if np.any(np.abs(sc - xs) > score_tol * np.abs(xs).max()):
            return False
        ds, di = np.diff(sc), np.diff(ids)
        if np.any((ds > 0) | ((ds == 0) & (di < 0))):
            return False
    return True
