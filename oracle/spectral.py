"""Eigenpairs, condition numbers and the CG convergence bound (oracle, FP64).

Sec. 3: eigenvalues of W lie in [-1, 1].  Sec. 4.1: U1, Lambda1 hold the
largest r eigenvalues (reading: algebraically largest) and their eigenvectors.
Sec. 4.4: Eq. 21 (CG bound phi_i), Eq. 22 (kappa of L_alpha(W)) and Eq. 23
(kappa of L_alpha(W_r) with W_r = W - U1 Lambda1 U1^T).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components


def eigh_desc(W) -> tuple[np.ndarray, np.ndarray]:
    """All eigenpairs of symmetric W, eigenvalues in descending order (dense)."""
    Wd = W.toarray() if sp.issparse(W) else np.asarray(W, dtype=np.float64)
    lam, U = np.linalg.eigh(Wd)
    return lam[::-1].copy(), U[:, ::-1].copy()


def eigenpairs(W, r: int) -> tuple[np.ndarray, np.ndarray]:
    """Largest r eigenvalues (descending) and eigenvectors of W (dense eigh)."""
    lam, U = eigh_desc(W)
    return lam[:r].copy(), U[:, :r].copy()


def deflated(W, U1: np.ndarray, lam1: np.ndarray) -> np.ndarray:
    """W_r = W - U1 Lambda1 U1^T as a dense matrix (Sec. 4.4)."""
    Wd = W.toarray() if sp.issparse(W) else np.asarray(W, dtype=np.float64)
    return Wd - (U1 * lam1) @ U1.T


def kappa_laplacian(alpha: float, lam_top: float, lam_min: float) -> float:
    """kappa(L_alpha(W_r)) = (1 - alpha lambda_n) / (1 - alpha lambda_{r+1})  (Eq. 22, 23)."""
    return (1.0 - alpha * lam_min) / (1.0 - alpha * lam_top)


def kappa_of(A) -> float:
    """2-norm condition number lambda_1(A) / lambda_n(A) of an SPD matrix (Sec. 4.4)."""
    Ad = A.toarray() if sp.issparse(A) else np.asarray(A, dtype=np.float64)
    ev = np.linalg.eigvalsh(Ad)
    return float(ev[-1] / ev[0])


def phi(kappa: float, i) -> np.ndarray:
    """CG bound phi_i(A) = 2 ((sqrt(kappa) - 1) / (sqrt(kappa) + 1))^i (Eq. 21)."""
    s = np.sqrt(kappa)
    return 2.0 * ((s - 1.0) / (s + 1.0)) ** np.asarray(i, dtype=np.float64)


def kappa_deflated(alpha: float, lam_next: float, lam_min: float) -> float:
    """kappa of L_alpha(W_r) when W_r keeps r zero eigenvalues (Sec. 4.4): its
    extremes are max(0, lambda_{r+1}) and min(0, lambda_n).  Equal to Eq. 23
    whenever lambda_{r+1} >= 0 >= lambda_n, the case the paper states."""
    return (1.0 - alpha * min(0.0, lam_min)) / (1.0 - alpha * max(0.0, lam_next))


def cg_iterations_bound(kappa: float, tol: float, kappa_res: float = 1.0) -> int:
    """Smallest i with sqrt(kappa_res) * phi_i(kappa) <= tol, by counting up
    (Eq. 21; kappa_res = 1: A-norm error reduced by tol; kappa_res = kappa(A):
    relative residual ||A e_i|| / ||A e_0|| <= tol, since that ratio is at most
    sqrt(kappa(A)) times the A-norm ratio)."""
    c = float(np.sqrt(kappa_res))
    i = 0
    while c * float(phi(kappa, i)) > tol:
        i += 1
    return i


def components(A) -> tuple[int, np.ndarray]:
    """Connected components of the graph of A (count, label per node)."""
    return connected_components(sp.csr_matrix(A), directed=False)


def a_norm(A, e: np.ndarray) -> float:
    """||e||_A = sqrt(e^T A e) (Sec. 4.4)."""
    return float(np.sqrt(e @ (A @ e)))
