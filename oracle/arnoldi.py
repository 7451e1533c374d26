"""Full block Arnoldi and the Galerkin solution (Section 2.1, Eq. (3.7)).

Test infrastructure: see oracle/__init__.py.

Block Arnoldi with modified block Gram-Schmidt against ALL previous blocks
(one reorthogonalisation pass for robustness; in exact arithmetic the second
pass adds zero), giving orthonormal U_{d+1}, V_{d+1} and block upper
Hessenberg H, G with A U_d = U_{d+1} H_(d+1 x d) (Eq. (2.1)).  The Galerkin
approximation X = U_d Y V_d^T solves H_d Y + Y G_d^T = E1 beta1 beta2^T E1^T,
and ||R||_F^2 = ||h_{d+1,d} E_d^T Y||^2 + ||Y E_d g_{d+1,d}^T||^2.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl

from .linalg import qr_pos, block_hessenberg


def block_arnoldi(op, C: np.ndarray, d: int, reorth: bool = True):
    """Orthonormal blocks U_1..U_{d+1}, Hessenberg blocks, beta (C = U_1 beta)."""
    C = np.asarray(C, dtype=np.float64)
    if C.ndim == 1:
        C = C[:, None]
    r = C.shape[1]
    U1, beta = qr_pos(C)
    blocks = {1: U1}
    H = {}
    for j in range(1, d + 1):
        W = op @ blocks[j]
        for _ in range(2 if reorth else 1):
            for i in range(1, j + 1):
                h = blocks[i].T @ W
                W = W - blocks[i] @ h
                H[(i, j)] = H.get((i, j), 0.0) + h
        Un, hn = qr_pos(W)
        blocks[j + 1] = Un
        H[(j + 1, j)] = hn
    return blocks, H, beta, r


def galerkin(A, BT, C1, C2, d: int, tol: float = 0.0, p: int = 1):
    """Full-Arnoldi Galerkin solution; checks every p up to d, stops at tol.

    Returns dict(d, X1=U_d Y (n1 x dr), X2=V_d (n2 x dr), Y, rho, rel).
    """
    Ub, H, b1, r = block_arnoldi(A, C1, d)
    Vb, G, b2, _ = block_arnoldi(BT, C2, d)
    nrm = np.linalg.norm(b1 @ b2.T)
    hist = []
    for dd in range(1, d + 1):
        if dd % p and dd != d:
            continue
        m = dd * r
        Hd = block_hessenberg(H, dd, r)
        Gd = block_hessenberg(G, dd, r)
        F = np.zeros((m, m))
        F[:r, :r] = b1 @ b2.T
        Y = sl.solve_sylvester(Hd[:m, :], Gd[:m, :].T, F)
        rho = np.sqrt(np.linalg.norm(Hd[m:, m - r:] @ Y[m - r:, :]) ** 2
                      + np.linalg.norm(Y[:, m - r:] @ Gd[m:, m - r:].T) ** 2)
        hist.append((dd, rho, rho / nrm))
        if rho / nrm < tol:
            break
    Ud = np.hstack([Ub[j] for j in range(1, dd + 1)])
    Vd = np.hstack([Vb[j] for j in range(1, dd + 1)])
    return dict(d=dd, Y=Y, X1=Ud @ Y, X2=Vd, hist=hist, rho=hist[-1][1], rel=hist[-1][2],
                U=Ud, V=Vd, H=H, G=G, beta1=b1, beta2=b2)


def memory_vectors_full(d: int, r: int) -> int:
    """Length-n vectors held by full Arnoldi: both bases, (d+1) r each
    (Table 1, the memory table of Section 5; the "Mem" column of the
    Section 6 tables)."""
    return 2 * (d + 1) * r


def memory_vectors_spkms(rank: int) -> int:
    """Length-n vectors of the s-PKSM solution factors X1, X2 (rank each),
    as the Section 6 tables count them."""
    return 2 * rank


def memory_vectors_tpkms(kA: int, kB: int, r: int) -> int:
    """Length-n vectors of the two truncated windows, k_A r + k_B r, as the
    t-PKSM table of Example 6.1 (Table 3) counts them."""
    return (kA + kB) * r
