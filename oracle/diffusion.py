"""Ranking vector x for observation y: every route of the paper (oracle, FP64).

Notation follows the paper: W is the normalised affinity (Sec. 3), alpha in
[0, 1), L_alpha(A) = (I - alpha A) / (1 - alpha) (Eq. 1),
h_alpha(A) = L_alpha(A)^-1 = (1 - alpha)(I - alpha A)^-1 (Eq. 3),
g_alpha(x) = h_alpha(x) - h_alpha(0) = (1 - alpha) alpha x / (1 - alpha x) (Eq. 16),
U1 (n x r) and Lambda1 (r) the largest r eigenpairs of W (Sec. 4.1).

Columns of a batch are solved one at a time with textbook CG (Hestenes-Stiefel)
from x0 = 0 (Sec. 4.4 takes e_0 = x*), stopping when ||r_i||_2 <= tol ||b||_2
or after max_iter operator applications.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def h_alpha(lam, alpha: float):
    """Scalar transfer function h_alpha(x) = (1 - alpha) / (1 - alpha x) (Sec. 3.2)."""
    lam = np.asarray(lam, dtype=np.float64)
    return (1.0 - alpha) / (1.0 - alpha * lam)


def g_alpha(lam, alpha: float):
    """Auxiliary g_alpha(x) = (1 - alpha) alpha x / (1 - alpha x) (Eq. 16)."""
    lam = np.asarray(lam, dtype=np.float64)
    return (1.0 - alpha) * alpha * lam / (1.0 - alpha * lam)


def closed_form(W, Y: np.ndarray, alpha: float) -> np.ndarray:
    """x = h_alpha(W) y = (1 - alpha)(I - alpha W)^-1 y by a dense solve (Eq. 3)."""
    Wd = W.toarray() if sp.issparse(W) else np.asarray(W, dtype=np.float64)
    n = Wd.shape[0]
    return (1.0 - alpha) * np.linalg.solve(np.eye(n) - alpha * Wd, np.asarray(Y, dtype=np.float64))


class CGResult:
    def __init__(self, x, iters, resnorms, converged):
        self.x = x
        self.iters = iters
        self.resnorms = resnorms      # ||r_i|| for i = 0..iters (recursive residual)
        self.converged = converged


def cg(apply_A, b: np.ndarray, tol: float, max_iter: int, x0=None, callback=None) -> CGResult:
    """Conjugate gradient for SPD A given as a black box z -> A z (Sec. 4.2, Sec. 4.4)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_A(x) if x0 is not None else b.copy()
    p = r.copy()
    rho = float(r @ r)
    bnorm = float(np.sqrt(b @ b))
    res = [np.sqrt(rho)]
    it = 0
    if callback is not None:
        callback(it, x)
    while it < max_iter and np.sqrt(rho) > tol * bnorm:
        q = apply_A(p)
        a = rho / float(p @ q)
        x = x + a * p
        r = r - a * q
        rho_new = float(r @ r)
        p = r + (rho_new / rho) * p
        rho = rho_new
        it += 1
        res.append(np.sqrt(rho))
        if callback is not None:
            callback(it, x)
    return CGResult(x, it, np.asarray(res), bool(np.sqrt(rho) <= tol * bnorm))


def pcg(apply_A, apply_Minv, b: np.ndarray, tol: float, max_iter: int) -> CGResult:
    """Preconditioned CG with SPD M^-1 given as a black box; stops on ||r|| <= tol ||b||."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    z = apply_Minv(r)
    p = z.copy()
    rho = float(r @ z)
    bnorm = float(np.sqrt(b @ b))
    res = [float(np.sqrt(r @ r))]
    it = 0
    while it < max_iter and res[-1] > tol * bnorm:
        q = apply_A(p)
        a = rho / float(p @ q)
        x = x + a * p
        r = r - a * q
        z = apply_Minv(r)
        rho_new = float(r @ z)
        p = z + (rho_new / rho) * p
        rho = rho_new
        it += 1
        res.append(float(np.sqrt(r @ r)))
    return CGResult(x, it, np.asarray(res), bool(res[-1] <= tol * bnorm))


def rows_matmul(W, Z, threads: int = 1) -> np.ndarray:
    """W @ Z, with the rows of W split into `threads` consecutive ranges done on
    threads.  Each output row is the same sum over the same entries in the same
    order as in W @ Z, so the result is identical; only the wall time differs."""
    if threads <= 1 or W.shape[0] < 4 * threads:
        return W @ Z
    from concurrent.futures import ThreadPoolExecutor
    Z = np.asarray(Z)
    bounds = np.linspace(0, W.shape[0], threads + 1).astype(np.int64)
    out = np.empty((W.shape[0],) + Z.shape[1:], dtype=np.result_type(W.dtype, Z.dtype))

    def part(t):
        out[bounds[t]:bounds[t + 1]] = W[bounds[t]:bounds[t + 1]] @ Z

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(part, range(threads)))
    return out


def cg_columns(apply_A, Bm, tol: float, max_iter: int, apply_Minv=None):
    """CG (PCG with apply_Minv) on every column of Bm, all columns at once.

    Each column runs the recurrences of `cg` / `pcg` above with its own step
    lengths and stops on its own ||r_j|| <= tol ||b_j|| (or max_iter); only the
    operator and preconditioner products are taken on the block of columns
    still running.  Returns (X, iters per column, recursive ||r_j|| / ||b_j||).
    """
    Bm = _columns(Bm)
    m = Bm.shape[1]
    X = np.zeros_like(Bm)
    R = Bm.copy()
    Z = R.copy() if apply_Minv is None else np.asarray(apply_Minv(R), dtype=np.float64)
    P = Z.copy()
    rho = np.einsum("ij,ij->j", R, Z)
    bnorm = np.linalg.norm(Bm, axis=0)
    rnorm = np.linalg.norm(R, axis=0)
    iters = np.zeros(m, dtype=np.int64)
    running = (rnorm > tol * bnorm) & (iters < max_iter)
    while running.any():
        c = np.where(running)[0]
        Pc = P[:, c]
        Qc = apply_A(Pc)
        a = rho[c] / np.einsum("ij,ij->j", Pc, Qc)
        X[:, c] += a * Pc
        Rc = R[:, c] - a * Qc
        R[:, c] = Rc
        Zc = Rc if apply_Minv is None else np.asarray(apply_Minv(Rc), dtype=np.float64)
        rho_new = np.einsum("ij,ij->j", Rc, Zc)
        P[:, c] = Zc + (rho_new / rho[c]) * Pc
        rho[c] = rho_new
        iters[c] += 1
        rnorm[c] = np.linalg.norm(Rc, axis=0)
        running = (rnorm > tol * bnorm) & (iters < max_iter)
    with np.errstate(invalid="ignore", divide="ignore"):
        rel = np.where(bnorm > 0, rnorm / np.where(bnorm > 0, bnorm, 1.0), 0.0)
    return X, iters, rel


def laplacian_op(W, alpha: float, threads: int = 1):
    """z -> L_alpha(W) z = (z - alpha W z) / (1 - alpha) (Eq. 1)."""
    return lambda z: (z - alpha * rows_matmul(W, z, threads)) / (1.0 - alpha)


def deflated_laplacian_op(W, U1: np.ndarray, lam1: np.ndarray, alpha: float):
    """Black box of Eq. 20: z -> (z - alpha (W z - U1 Lambda1 U1^T z)) / (1 - alpha).

    The low-rank product is taken right to left: U1 (Lambda1 (U1^T z)).
    """
    return lambda z: (z - alpha * ((W @ z) - U1 @ (lam1 * (U1.T @ z)))) / (1.0 - alpha)


def _columns(Y):
    Y = np.asarray(Y, dtype=np.float64)
    return Y[:, None] if Y.ndim == 1 else Y


def temporal(W, Y, alpha: float, tol: float, max_iter: int):
    """Temporal filtering: solve L_alpha(W) x = y by CG, per column (Eq. 2)."""
    Y = _columns(Y)
    A = laplacian_op(W, alpha)
    out = [cg(A, Y[:, j], tol, max_iter) for j in range(Y.shape[1])]
    return np.stack([o.x for o in out], 1), [o.iters for o in out], out


def spectral(U: np.ndarray, lam: np.ndarray, Y, alpha: float) -> np.ndarray:
    """Spectral filtering x = U h_alpha(Lambda) U^T y, right to left (Eq. 4)."""
    Y = _columns(Y)
    return U @ (h_alpha(lam, alpha)[:, None] * (U.T @ Y))


def spectral_term(U1: np.ndarray, lam1: np.ndarray, Y, alpha: float) -> np.ndarray:
    """x^s = U1 g_alpha(Lambda1) U1^T y (Eq. 18)."""
    Y = _columns(Y)
    return U1 @ (g_alpha(lam1, alpha)[:, None] * (U1.T @ Y))


def hybrid(W, U1: np.ndarray, lam1: np.ndarray, Y, alpha: float, tol: float, max_iter: int):
    """The paper's hybrid filtering (Form P): x = x^s + x^t (Eq. 17).

    x^s by Eq. 18; x^t by CG on L_alpha(W - U1 Lambda1 U1^T) x^t = y using the
    black box of Eq. 20 (Eq. 19).  Returns (x, iters, x^s, x^t).
    """
    Y = _columns(Y)
    xs = spectral_term(U1, lam1, Y, alpha)
    A = deflated_laplacian_op(W, U1, lam1, alpha)
    res = [cg(A, Y[:, j], tol, max_iter) for j in range(Y.shape[1])]
    xt = np.stack([o.x for o in res], 1)
    return xs + xt, [o.iters for o in res], xs, xt


def hybrid_projected(W, U1: np.ndarray, lam1: np.ndarray, Y, alpha: float, tol: float, max_iter: int):
    """Projected hybrid (Form N): x = U1 h(Lambda1) U1^T y + (1 - alpha) x2 with
    (I - alpha (W - U1 Lambda1 U1^T)) x2 = (I - U1 U1^T) y.

    Equal to Eq. 17 in exact arithmetic: by Eq. 5 the temporal operator maps
    range(U2) to itself, so x2 = U2 (I - alpha Lambda2)^-1 U2^T y.
    """
    Y = _columns(Y)
    C = U1.T @ Y
    xs = U1 @ (h_alpha(lam1, alpha)[:, None] * C)
    B2 = Y - U1 @ C
    A = lambda z: z - alpha * ((W @ z) - U1 @ (lam1 * (U1.T @ z)))  # noqa: E731
    res = [cg(A, B2[:, j], tol, max_iter) for j in range(Y.shape[1])]
    x2 = np.stack([o.x for o in res], 1)
    return xs + (1.0 - alpha) * x2, [o.iters for o in res]


def preconditioner_weights(lam1: np.ndarray, alpha: float) -> np.ndarray:
    """D = alpha l / (1 - alpha l) with l = max(lambda, 0): M^-1 = I + U1 D U1^T."""
    lt = np.maximum(np.asarray(lam1, dtype=np.float64), 0.0)
    return alpha * lt / (1.0 - alpha * lt)


def hybrid_pcg(W, U1: np.ndarray, lam1: np.ndarray, Y, alpha: float, tol: float, max_iter: int):
    """Spectrally preconditioned hybrid (Form S): PCG on L_alpha(W) x = y with
    M^-1 = I + U1 diag(alpha l / (1 - alpha l)) U1^T.

    With exact eigenpairs M^-1 L_alpha(W) has eigenvalues 1/(1 - alpha) (for the
    r removed ones) and (1 - alpha lambda_j)/(1 - alpha) for j > r, so its
    condition number is Eq. 23's; for any U1 the iteration still converges to
    h_alpha(W) y because M^-1 stays symmetric positive definite.
    """
    Y = _columns(Y)
    D = preconditioner_weights(lam1, alpha)
    A = laplacian_op(W, alpha)
    Minv = lambda z: z + U1 @ (D * (U1.T @ z))  # noqa: E731
    res = [pcg(A, Minv, Y[:, j], tol, max_iter) for j in range(Y.shape[1])]
    return np.stack([o.x for o in res], 1), [o.iters for o in res]


def neumann(W, Y, alpha: float, terms: int) -> np.ndarray:
    """(1 - alpha) sum_{i < terms} alpha^i W^i y: the series of Eq. 3 (Appendix A, Eq. 24)."""
    Y = _columns(Y)
    acc = np.zeros_like(Y)
    t = Y.copy()
    for _ in range(terms):
        acc += t
        t = alpha * (W @ t)
    return (1.0 - alpha) * acc
