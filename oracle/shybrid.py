"""SHybrid: sparsified spectral embedding U1 (oracle).

Sec. 5.3: the smallest values of U1 are set to zero until a desired sparsity is
reached.  Reading: "smallest" is by absolute value over the whole n x r matrix;
equal magnitudes are dropped in row-major order (the later entry is dropped
first), so the kept set is unique.
"""
from __future__ import annotations

import numpy as np


def sparsify(U1: np.ndarray, sparsity: float) -> np.ndarray:
    """Zero the round(sparsity * n * r) entries of smallest |U1_ij|."""
    U = np.asarray(U1, dtype=np.float64)
    flat = U.ravel()
    drop = int(round(sparsity * flat.size))
    order = np.lexsort((-np.arange(flat.size), np.abs(flat)))  # ascending |u|, later index first
    out = flat.copy()
    out[order[:drop]] = 0.0
    return out.reshape(U.shape)
