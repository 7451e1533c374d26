"""Algorithm 2 (t-PKSM): truncated Arnoldi without sketching.

Test infrastructure: see oracle/__init__.py.

Truncated block Arnoldi with windows k_A, k_B (modified Gram-Schmidt over
the last k blocks), projected equation H_d Y + Y G_d^T = E1 beta1 beta2^T E1^T
(Section 3), and the residual bound of Proposition 3.1 (Eq. (3.2)):
    rho = sqrt(dr) (||Y E_d g_{d+1,d}^T||_F + ||h_{d+1,d} E_d^T Y||_F).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl

from .linalg import qr_pos, right_solve_upper, block_hessenberg


def _truncated(op, C, k, d):
    """Algorithm 2's truncated block Arnoldi (Appendix A): A U_j is
    orthogonalised by modified Gram-Schmidt against U_{j-k+1}, ..., U_j only,
    then U_{j+1} h_{j+1,j} is its positive-diagonal skinny QR.  Returns all
    blocks {j: U_j}, the banded H {(i, j): h_ij} and beta (C = U_1 beta)."""
    U1, beta = qr_pos(C)
    blocks = {1: U1}
    H = {}
    for j in range(1, d + 1):
        W = op @ blocks[j]
        for i in range(max(1, j - k + 1), j + 1):
            h = blocks[i].T @ W
            W = W - blocks[i] @ h
            H[(i, j)] = h
        Un, hn = qr_pos(W)
        blocks[j + 1] = Un
        H[(j + 1, j)] = hn
    return blocks, H, beta


def tpkms(A, BT, C1, C2, *, kA: int, kB: int, tol: float, maxit: int, p: int = 1):
    """Run Algorithm 2 (t-PKSM, Appendix A): truncated bases of K_d(A, C1)
    and K_d(B^T, C2) with windows k_A and k_B, then every p iterations the
    projected equation H_d Y + Y G_d^T = E_1 beta_1 beta_2^T E_1^T with the
    banded H_d, G_d, and the residual bound of Proposition 3.1 (Eq. (3.2)),
    tested against tol relative to ||beta_1 beta_2^T||_F.  Returns
    X1 = U_d Y and X2 = V_d (Y not truncated), the history and the bases."""
    C1 = np.atleast_2d(np.asarray(C1, dtype=np.float64).T).T
    C2 = np.atleast_2d(np.asarray(C2, dtype=np.float64).T).T
    r = C1.shape[1]
    Ub, H, b1 = _truncated(A, C1, kA, maxit)
    Vb, G, b2 = _truncated(BT, C2, kB, maxit)
    nrm = np.linalg.norm(b1 @ b2.T)
    hist = []
    for d in range(1, maxit + 1):
        if d % p and d != maxit:
            continue
        m = d * r
        Hd = block_hessenberg(H, d, r)
        Gd = block_hessenberg(G, d, r)
        F = np.zeros((m, m))
        F[:r, :r] = b1 @ b2.T
        Y = sl.solve_sylvester(Hd[:m, :], Gd[:m, :].T, F)
        rho = np.sqrt(m) * (np.linalg.norm(Y[:, m - r:] @ Gd[m:, m - r:].T)
                            + np.linalg.norm(Hd[m:, m - r:] @ Y[m - r:, :]))
        hist.append((d, rho, rho / nrm))
        if rho / nrm < tol:
            break
    Ud = np.hstack([Ub[j] for j in range(1, d + 1)])
    Vd = np.hstack([Vb[j] for j in range(1, d + 1)])
    return dict(d=d, Y=Y, X1=Ud @ Y, X2=Vd, hist=hist, U=Ud, V=Vd, H=H, G=G)
