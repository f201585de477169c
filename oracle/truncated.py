"""Temporal filtering on a truncated graph, "Temporal†" (oracle, FP64).

Sec. 3.1 and Sec. 5.1 (Table 1, Fig. 5): at large scale the temporal system is
solved only on a shortlist S of the query's nearest database items: the rows
and columns of the affinity for S are kept, the subgraph is normalised again
by its own degrees, and the linear system of Eq. 2 is solved there, so that
only the shortlist is re-ranked.

Readings (the paper defers to its reference for the details):
* the affinity A (not W) is restricted and normalised again,
  W_S = D_S^-1/2 A_SS D_S^-1/2 with D_S = diag(A_SS 1) -- the rule of Sec. 3
  applied to the subgraph; a node with no edge inside S gets D^-1/2 := 0;
* y_S is y restricted to S (observations outside S are dropped);
* the shortlist is the s database items of largest similarity to the query
  descriptor, ties to the smaller id; x_S is returned in shortlist order.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import diffusion


def shortlist(X: np.ndarray, q: np.ndarray, s: int) -> np.ndarray:
    """Ids of the s largest q^T x_i, descending, equal similarities to the smaller id."""
    sims = np.asarray(X, dtype=np.float64) @ np.asarray(q, dtype=np.float64)
    order = np.lexsort((np.arange(sims.size), -sims))
    return order[:s].astype(np.int64)


def subsystem(A: sp.csr_matrix, S: np.ndarray) -> tuple[sp.csr_matrix, np.ndarray]:
    """(W_S, D_S^-1/2) of the subgraph on the ids S, in the order of S."""
    S = np.asarray(S, dtype=np.int64)
    A_SS = sp.csr_matrix(A)[S][:, S].tocsr()
    d = np.asarray(A_SS.sum(axis=1)).ravel()
    dinv = np.zeros_like(d)
    nz = d > 0
    dinv[nz] = 1.0 / np.sqrt(d[nz])
    Dm = sp.diags(dinv)
    return (Dm @ A_SS @ Dm).tocsr(), dinv


def temporal_truncated(A: sp.csr_matrix, S: np.ndarray, y: np.ndarray, alpha: float, tol: float, max_iter: int):
    """x_S solving L_alpha(W_S) x_S = y_S by CG (Eq. 2 on the subgraph); (x_S, iterations)."""
    W_S, _ = subsystem(A, S)
    y_S = np.asarray(y, dtype=np.float64)[np.asarray(S, dtype=np.int64)]
    res = diffusion.cg(diffusion.laplacian_op(W_S, alpha), y_S, tol, max_iter)
    return res.x, res.iters
