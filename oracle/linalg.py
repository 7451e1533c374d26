"""Small dense helpers shared inside the oracle (FP64, NumPy/SciPy)."""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl


def qr_pos(M: np.ndarray):
    """Reduced QR with a positive diagonal in R (unique for full column rank).

    Householder QR from LAPACK, then column/row signs flipped so R_ii > 0
    (the convention that makes h_{d+1,d}, tau_d and beta unique).
    """
    Q, R = np.linalg.qr(np.asarray(M, dtype=np.float64), mode="reduced")
    sgn = np.sign(np.diag(R))
    sgn[sgn == 0] = 1.0
    return Q * sgn[None, :], R * sgn[:, None]


def right_solve_upper(M: np.ndarray, T: np.ndarray) -> np.ndarray:
    """M T^{-1} for upper triangular T (solve X T = M)."""
    return sl.solve_triangular(T, M.T, trans="T", lower=False).T


def left_solve_upper(T: np.ndarray, M: np.ndarray) -> np.ndarray:
    """T^{-1} M for upper triangular T."""
    return sl.solve_triangular(T, M, lower=False)


def block_hessenberg(blocks: dict, d: int, r: int) -> np.ndarray:
    """Dense (d+1)r x dr matrix from blocks {(i, j): r x r} (1-based)."""
    H = np.zeros(((d + 1) * r, d * r))
    for (i, j), h in blocks.items():
        if j <= d and i <= d + 1:
            H[(i - 1) * r:i * r, (j - 1) * r:j * r] = h
    return H
