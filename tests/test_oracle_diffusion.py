"""Pins for oracle.diffusion: closed form, series, special cases r=0 and r=n, invariants."""
import numpy as np
import pytest

from oracle import diffusion as D
from oracle import spectral as S
from oracle import observe


def _y(n, B, seed=0, nnz=5):
    rng = np.random.default_rng(seed)
    Y = np.zeros((n, B))
    for j in range(B):
        idx = rng.choice(n, nnz, replace=False)
        Y[idx, j] = rng.uniform(0.1, 1.0, nnz)
    return Y


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("alpha,terms", [(0.5, 80), (0.9, 450), (0.99, 4000)])
def test_closed_form_equals_neumann_series(small_graph, alpha, terms):
    # Eq. 3 by a dense solve versus the power series of (I - alpha W)^-1.
    W = small_graph["W"]
    Y = _y(60, 3)
    assert _rel(D.closed_form(W, Y, alpha), D.neumann(W, Y, alpha, terms)) < 1e-12


def test_temporal_cg_reaches_closed_form(small_graph):
    W = small_graph["W"]
    Y = _y(60, 4, 1)
    x, iters, _ = D.temporal(W, Y, 0.99, 1e-14, 1000)
    assert _rel(x, D.closed_form(W, Y, 0.99)) < 1e-11
    assert all(i > 1 for i in iters)


@pytest.mark.parametrize("r", [0, 1, 2, 5, 17, 30, 59, 60])
def test_hybrid_every_rank_equals_closed_form(small_graph, r):
    # Theorem 1 / Eq. 17-20: the hybrid is exact for every r with exact eigenpairs.
    W = small_graph["W"]
    Y = _y(60, 3, 2)
    lam, U = S.eigenpairs(W, r)
    x, _, xs, xt = D.hybrid(W, U, lam, Y, 0.99, 1e-14, 2000)
    assert _rel(x, D.closed_form(W, Y, 0.99)) < 1e-10


def test_r0_is_temporal_iterate_for_iterate(small_graph):
    W = small_graph["W"]
    Y = _y(60, 2, 3)
    U0, l0 = np.zeros((60, 0)), np.zeros(0)
    x_h, it_h, xs, _ = D.hybrid(W, U0, l0, Y, 0.99, 1e-8, 500)
    x_t, it_t, _ = D.temporal(W, Y, 0.99, 1e-8, 500)
    assert it_h == it_t
    assert np.array_equal(x_h, x_t)
    assert np.all(xs == 0)


def test_r_equals_n_is_spectral(small_graph):
    # With all n eigenpairs W_r = 0, L_alpha(W_r) = I / (1 - alpha): one CG step,
    # x^t = (1 - alpha) y and x = U h(Lambda) U^T y (Eq. 4).
    W = small_graph["W"]
    Y = _y(60, 3, 4)
    lam, U = S.eigenpairs(W, 60)
    x, iters, xs, xt = D.hybrid(W, U, lam, Y, 0.99, 1e-12, 50)
    assert all(i == 1 for i in iters)
    assert np.allclose(xt, 0.01 * Y, atol=1e-13)
    assert _rel(x, D.spectral(U, lam, Y, 0.99)) < 1e-11
    assert _rel(D.spectral(U, lam, Y, 0.99), D.closed_form(W, Y, 0.99)) < 1e-11


@pytest.mark.parametrize("r", [0, 3, 12, 40])
def test_projected_and_preconditioned_forms(small_graph, r):
    W = small_graph["W"]
    Y = _y(60, 3, 5)
    lam, U = S.eigenpairs(W, r)
    ref = D.closed_form(W, Y, 0.99)
    xn, _ = D.hybrid_projected(W, U, lam, Y, 0.99, 1e-14, 2000)
    xs, _ = D.hybrid_pcg(W, U, lam, Y, 0.99, 1e-14, 2000)
    assert _rel(xn, ref) < 1e-10
    assert _rel(xs, ref) < 1e-10


def test_preconditioned_form_is_exact_for_any_basis(small_graph):
    # Form S converges to x* even when U1 is not made of eigenvectors.
    W = small_graph["W"]
    Y = _y(60, 2, 6)
    lam, U = S.eigenpairs(W, 10)
    rng = np.random.default_rng(0)
    Up = U + 1e-2 * rng.standard_normal(U.shape)
    x, _ = D.hybrid_pcg(W, Up, lam, Y, 0.99, 1e-14, 2000)
    assert _rel(x, D.closed_form(W, Y, 0.99)) < 1e-10
    # ...while the paper's form with the same perturbed basis is off to first order.
    xp, *_ = D.hybrid(W, Up, lam, Y, 0.99, 1e-14, 2000)
    assert _rel(xp, D.closed_form(W, Y, 0.99)) > 1e-4


def test_fewer_iterations_with_more_eigenpairs(small_graph):
    W = small_graph["W"]
    Y = _y(60, 2, 7)
    its = []
    for r in (0, 4, 20):
        lam, U = S.eigenpairs(W, r)
        _, it, _, _ = D.hybrid(W, U, lam, Y, 0.99, 1e-8, 500)
        its.append(max(it))
    assert its[0] > its[1] >= its[2]


def test_solution_invariants(small_graph):
    # Neumann series with W >= 0: x* >= (1 - alpha) y >= 0 elementwise.
    # sqrt(d) is the eigenvalue-1 eigenvector and h(1) = 1: sqrt(d)^T x* = sqrt(d)^T y.
    W, A = small_graph["W"], small_graph["A"]
    Y = _y(60, 4, 8)
    x = D.closed_form(W, Y, 0.99)
    assert np.all(x >= 0.01 * Y - 1e-15)
    sd = np.sqrt(np.asarray(A.sum(1)).ravel())
    ncomp, lab = S.components(A)
    for c in range(ncomp):
        m = lab == c
        assert np.allclose(sd[m] @ x[m], sd[m] @ Y[m], rtol=1e-10)


def test_transfer_functions():
    lam = np.array([-1.0, 0.0, 0.3, 1.0])
    assert np.allclose(D.h_alpha(lam, 0.99), [0.01 / 1.99, 0.01, 0.01 / 0.703, 1.0])
    assert np.allclose(D.g_alpha(lam, 0.99), D.h_alpha(lam, 0.99) - 0.01)
    assert np.allclose(D.preconditioner_weights(lam, 0.99), [0, 0, 0.297 / 0.703, 99.0])


def test_spectral_term_uses_g_not_h(small_graph):
    W = small_graph["W"]
    Y = _y(60, 1, 9)
    lam, U = S.eigenpairs(W, 8)
    xs = D.spectral_term(U, lam, Y, 0.99)
    full = D.spectral(U, lam, Y, 0.99)
    # U h U^T y - U g U^T y = h(0) U U^T y = (1 - alpha) U U^T y
    assert np.allclose(full - xs, 0.01 * U @ (U.T @ Y), atol=1e-14)


def test_observation_feeds_dense(small_graph):
    ptr, idx, val = observe.observe(small_graph["X"], small_graph["X"][:2] * 0.9, 4)
    Y = observe.dense(60, ptr, idx, val)
    assert Y.shape == (60, 2) and np.count_nonzero(Y) <= 8


def test_rows_matmul_is_the_plain_product(small_graph):
    # the row-split product computes each row exactly as W @ Z does
    W = small_graph["W"]
    Z = np.random.default_rng(4).standard_normal((60, 5))
    for t in (1, 2, 3, 8):
        assert np.array_equal(D.rows_matmul(W, Z, t), W @ Z)
        assert np.array_equal(D.laplacian_op(W, 0.9, t)(Z), D.laplacian_op(W, 0.9)(Z))


@pytest.mark.parametrize("tol", [1e-4, 1e-8, 1e-13])
def test_cg_columns_equals_column_by_column_cg(small_graph, tol):
    # all columns at once, each with its own step lengths and stopping: the
    # iteration counts and iterates of the one-column CG / PCG (Sec. 4.4)
    W = small_graph["W"]
    Y = _y(60, 5, 7, nnz=3)
    Y[:, 2] *= 1e-3                       # columns of very different scale
    A = D.laplacian_op(W, 0.99)
    X, it, rel = D.cg_columns(A, Y, tol, 500)
    for j in range(Y.shape[1]):
        ref = D.cg(A, Y[:, j], tol, 500)
        assert it[j] == ref.iters
        assert np.linalg.norm(X[:, j] - ref.x) <= 1e-12 * np.linalg.norm(ref.x)
        assert rel[j] <= tol
    lam, U = S.eigenpairs(W, 7)
    Dw = D.preconditioner_weights(lam, 0.99)
    Minv = lambda z: z + U @ (Dw[:, None] * (U.T @ z)) if np.ndim(z) == 2 else z + U @ (Dw * (U.T @ z))  # noqa: E731
    Xp, itp, _ = D.cg_columns(A, Y, tol, 500, apply_Minv=Minv)
    for j in range(Y.shape[1]):
        ref = D.pcg(A, Minv, Y[:, j], tol, 500)
        assert itp[j] == ref.iters
        assert np.linalg.norm(Xp[:, j] - ref.x) <= 1e-12 * np.linalg.norm(ref.x)
    if tol < 1e-12:
        assert _rel(X, D.closed_form(W, Y, 0.99)) < 1e-11
