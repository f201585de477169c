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
import test_oracle_truncated as TT
from oracle import diffusion as D
from oracle import general as GE
from oracle import graph as G
from oracle import observe as O
from oracle import rank as R
from oracle import shybrid as SH
from oracle import spectral as SP
from oracle import truncated as T


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


def _subsystem_not_renormalised(A, S):
    W, dinv = G.normalize(A)
    S = np.asarray(S, dtype=np.int64)
    return W[S][:, S].tocsr(), dinv[S]


def _kappa_unclamped(alpha, lam_next, lam_min):
    return (1.0 - alpha * lam_min) / (1.0 - alpha * lam_next)


def _bound_one_short(kappa, tol, kappa_res=1.0):
    i = 0
    while np.sqrt(kappa_res) * float(SP.phi(kappa, i)) > tol:
        i += 1
    return max(i - 1, 0)


def _sparsify_earlier_first(U1, sparsity):
    U = np.asarray(U1, dtype=np.float64)
    flat = U.ravel()
    drop = int(round(sparsity * flat.size))
    order = np.lexsort((np.arange(flat.size), np.abs(flat)))
    out = flat.copy()
    out[order[:drop]] = 0.0
    return out.reshape(U.shape)


def _poly_coefficients_reversed(apply_A, coeffs, y):
    acc = np.zeros_like(np.asarray(y, dtype=np.float64))
    for c in list(coeffs):
        acc = apply_A(acc) + c * y
    return acc


def _regional_first_region_only(Xdb, Q, regions, k_y, gamma=3.0):
    p, i, v = O.observe(Xdb, Q[::regions], k_y, gamma)
    return p, i, v


def _ranks_match_positionwise_only(ids, ids_ref, score_ref, tie, scores=None, x=None, score_tol=0.0):
    for a, b in zip(ids, ids_ref):
        if a != b and abs(score_ref[a] - score_ref[b]) > tie:
            return False
    return True


def _cg_columns_shared_step(apply_A, Bm, tol, max_iter, apply_Minv=None):
    # one step length for every column (the first column's): a plausible
    # mistake when vectorising CG over a block
    Bm = np.asarray(Bm, dtype=np.float64)
    X = np.zeros_like(Bm)
    R = Bm.copy()
    P = R.copy()
    rho = np.einsum("ij,ij->j", R, R)
    bn = np.linalg.norm(Bm, axis=0)
    it = 0
    with np.errstate(all="ignore"):
        while it < max_iter and np.any(np.linalg.norm(R, axis=0) > tol * bn):
            Q = apply_A(P)
            a = rho[0] / float(P[:, 0] @ Q[:, 0])
            X += a * P
            R -= a * Q
            rn = np.einsum("ij,ij->j", R, R)
            P = R + (rn / rho) * P
            rho = rn
            it += 1
    m = Bm.shape[1]
    return X, np.full(m, it), np.linalg.norm(R, axis=0) / bn


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
    ("truncated subgraph not renormalised", T, "subsystem", _subsystem_not_renormalised,
     lambda g: TT.test_matches_dense_solve_built_by_loops(TT.make_g80())),
    ("deflated kappa unclamped", SP, "kappa_deflated", _kappa_unclamped,
     lambda g: TS.test_kappa_deflated_against_dense(g)),
    ("iteration bound one short", SP, "cg_iterations_bound", _bound_one_short,
     lambda g: TS.test_iteration_bound_holds_for_cg_and_pcg(g, 1e-4)),
    ("sparsify drops the earlier tie", SH, "sparsify", _sparsify_earlier_first,
     lambda g: TS.test_sparsify_keeps_largest_magnitudes()),
    ("regional observation from one region", O, "observe_regional", _regional_first_region_only,
     lambda g: TG.test_observe_regional_is_the_sum_of_region_observations()),
    ("polynomial coefficients reversed", GE, "poly_apply", _poly_coefficients_reversed,
     lambda g: TS.test_poly_apply_against_dense_spectral_evaluation(g)),
    ("ranking check position-wise only", R, "ranks_match", _ranks_match_positionwise_only,
     lambda g: TS.test_ranks_match_rejects_invalid_rankings()),
    ("block CG with one step length", D, "cg_columns", _cg_columns_shared_step,
     lambda g: TD.test_cg_columns_equals_column_by_column_cg(g, 1e-8)),
]


@pytest.mark.parametrize("name,mod,attr,bad,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_mutant(small_graph, monkeypatch, name, mod, attr, bad, pin):
    pin(small_graph)                      # the pin passes on the real oracle
    monkeypatch.setattr(mod, attr, bad)
    with pytest.raises(AssertionError):
        pin(small_graph)
