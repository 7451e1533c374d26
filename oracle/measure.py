"""Gauge-free comparisons of low-rank factorisations (test infrastructure).

X = X1 X2^T is never formed.  ||X1 X2^T - Z1 Z2^T||_F is computed from
Householder QRs of the stacked factors, [X1, -Z1] = Qa Ra, [X2, Z2] = Qb Rb,
so that the difference equals Qa (Ra Rb^T) Qb^T and its Frobenius norm is
||Ra Rb^T||_F -- no Gram-trace cancellation, accurate to ~u relative.
The true residual R = A X + X B - C1 C2^T has the factored form
[A X1, X1, -C1] [X2, B^T X2, C2]^T and is measured the same way.
"""
from __future__ import annotations

import numpy as np


def lowrank_fro(L: np.ndarray, R: np.ndarray) -> float:
    """||L R^T||_F."""
    if L.shape[1] == 0:
        return 0.0
    _, Ra = np.linalg.qr(L, mode="reduced")
    _, Rb = np.linalg.qr(R, mode="reduced")
    return float(np.linalg.norm(Ra @ Rb.T))


def lowrank_diff_fro(X1, X2, Z1, Z2) -> float:
    """||X1 X2^T - Z1 Z2^T||_F."""
    return lowrank_fro(np.hstack([X1, -Z1]), np.hstack([X2, Z2]))


def rel_error(X1, X2, Z1, Z2) -> float:
    """||X - Z||_F / ||Z||_F for X = X1 X2^T, Z = Z1 Z2^T."""
    return lowrank_diff_fro(X1, X2, Z1, Z2) / lowrank_fro(Z1, Z2)


def true_residual(A, B, C1, C2, X1, X2) -> float:
    """||A X + X B - C1 C2^T||_F / ||C1 C2^T||_F with X = X1 X2^T."""
    BT = B.T
    L = np.hstack([A @ X1, X1, -C1])
    R = np.hstack([X2, BT @ X2, C2])
    return lowrank_fro(L, R) / lowrank_fro(C1, C2)


def probe_errors(X1, X2, Z1, Z2, count: int = 16, seed: int = 12345) -> float:
    """max over Gaussian probes w of ||(X - Z) w|| / ||Z w|| and with w^T."""
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(count):
        w = rng.standard_normal(X2.shape[0])
        a = X1 @ (X2.T @ w) - Z1 @ (Z2.T @ w)
        worst = max(worst, float(np.linalg.norm(a) / np.linalg.norm(Z1 @ (Z2.T @ w))))
        w = rng.standard_normal(X1.shape[0])
        a = X2 @ (X1.T @ w) - Z2 @ (Z1.T @ w)
        worst = max(worst, float(np.linalg.norm(a) / np.linalg.norm(Z2 @ (Z1.T @ w))))
    return worst
