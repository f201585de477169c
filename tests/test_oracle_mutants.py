"""Planted mistakes in the oracle must make at least one pin fail.

Each case swaps one oracle function for a plausibly wrong variant (a dropped
factor, a sign flip, a wrong index rule) and runs the pin that should catch
it.  Everything here runs on the CPU and touches only the oracle.
"""
import numpy as np
import pytest

import test_oracle_diffusion as TD
import test_oracle_graph as TG
import test_oracle_spectral as TS
from oracle import diffusion as D
from oracle import graph as G
from oracle import rank as R


def _g_no_one_minus_alpha(lam, alpha):
    lam = np.asarray(lam, dtype=np.float64)
    return alpha * lam / (1.0 - alpha * lam)


def _deflated_sign_flip(W, U1, lam1, alpha):
    return lambda z: (z - alpha * ((W @ z) + U1 @ (lam1 * (U1.T @ z)))) / (1.0 - alpha)


def _closed_form_no_scale(W, Y, alpha):
    Wd = W.toarray() if hasattr(W, "toarray") else np.asarray(W)
    return np.linalg.solve(np.eye(Wd.shape[0]) - alpha * Wd, Y)


def _laplacian_no_division(W, alpha):
    return lambda z: z - alpha * (W @ z)


def _normalize_random_walk(A):
    d = np.asarray(A.sum(axis=1)).ravel()
    import scipy.sparse as sp
    W = (sp.diags(1.0 / d) @ A).tocsr()
    return W, 1.0 / np.sqrt(d)


def _topk_larger_id_first(x, K):
    x = np.asarray(x)
    order = np.lexsort((-np.arange(x.size), -x))[:K]
    return order, x[order]


def _knn_with_self(X, rows, k):
    X = np.asarray(X, dtype=np.float64)
    idx = np.empty((len(rows), k), dtype=np.int64)
    sim = np.empty((len(rows), k))
    for t, i in enumerate(rows):
        s = X @ X[i]
        order = np.lexsort((np.arange(len(X)), -s))[:k]
        idx[t], sim[t] = order, s[order]
    return idx, sim


def _g_transposed_basis(U1, lam1, Y, alpha):
    Y = np.asarray(Y, dtype=np.float64)
    Y = Y[:, None] if Y.ndim == 1 else Y
    return U1 @ (D.g_alpha(lam1, alpha)[:, None] * (U1.T @ Y))[::-1]


MUTANTS = [
    ("g drops (1-alpha)", D, "g_alpha", _g_no_one_minus_alpha,
     lambda g: TD.test_hybrid_every_rank_equals_closed_form(g, 5)),
    ("black box sign flip", D, "deflated_laplacian_op", _deflated_sign_flip,
     lambda g: TD.test_hybrid_every_rank_equals_closed_form(g, 5)),
    ("closed form unscaled", D, "closed_form", _closed_form_no_scale,
     lambda g: TD.test_closed_form_equals_neumann_series(g, 0.9, 450)),
    ("laplacian undivided", D, "laplacian_op", _laplacian_no_division,
     lambda g: TD.test_temporal_cg_reaches_closed_form(g)),
    ("random-walk normalisation", G, "normalize", _normalize_random_walk,
     lambda g: TG.test_graph_invariants({**g, "W": G.normalize(g["A"])[0]})),
    ("ties to the larger id", R, "topk", _topk_larger_id_first,
     lambda g: TS.test_topk_matches_python_sort()),
    ("self in neighbour list", G, "knn_rows", _knn_with_self,
     lambda g: TG.test_adjacency_matches_loops("union")),
    ("spectral term rows permuted", D, "spectral_term", _g_transposed_basis,
     lambda g: TD.test_hybrid_every_rank_equals_closed_form(g, 17)),
]


@pytest.mark.parametrize("name,mod,attr,bad,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_mutant(small_graph, monkeypatch, name, mod, attr, bad, pin):
    pin(small_graph)                      # the pin passes on the real oracle
    monkeypatch.setattr(mod, attr, bad)
    with pytest.raises(AssertionError):
        pin(small_graph)
