"""Algorithm 1 (s-PKSM) of the paper, step by step, in FP64 on the CPU.

Test infrastructure: see oracle/__init__.py.

The method solves A X + X B = C1 C2^T (Eq. (1.1)) by truncated block Arnoldi
(Eq. (2.4)) on K_d(A, C1) and K_d(B^T, C2), whitens the non-orthogonal bases
through the QR factorisations of their sketches (Proposition 2.1, Eqs. (2.5)-(2.6)),
solves the sketched Galerkin problem (Eq. (3.4)) and estimates the sketched
residual norm (Eq. (3.5)); the factors are recovered by a second Arnoldi sweep
that replays the stored coefficients (Section 5).

Readings taken where the paper is garbled or silent (each pinned by a test):
  * T_{U,1} is the R factor of S_U U_1, so beta_1 = T_{U,1} ell with
    U_1 ell = C1 (Algorithm 1 sets T_{U,1} = beta_1, which contradicts
    C1 = Uhat_d E_1 beta_1 of Eq. (3.4) unless ell = I); C2 is sketched by
    S_V, not S_U.
  * The residual estimate (Eq. (3.5), Algorithm 1) uses the whitened
    subdiagonal hhat = tau_{d+1} h_{d+1,d} tau_d^{-1} (and ghat likewise),
    which is what Proposition 2.1 times T_d^{-1} gives and what the (d+1, d)
    block of the Section 5 bordering formula is.
  * The Section 5 bordering formula's last term of Hhat_new carries
    tau_{d+1}^{-1}, not tau_d^{-1} (direct expansion of T H T^{-1}).
  * Stopping test relative: rho / ||beta_1 beta_2^T||_F < tol.
  * Truncation of Y: SVD, keep sigma_i > trunc_tol * sigma_1,
    Y1 = P Sigma^{1/2}, Y2 = Q Sigma^{1/2}; X1 = U_d T_U^{-1} Y1,
    X2 = V_d T_V^{-1} Y2.
  * If maxit is reached between checks, one last check is made at maxit.
  * Orthogonalisation is modified Gram-Schmidt over the window, as written
    in Algorithm 1; the new block is U_{d+1} = U~ h_{d+1,d}^{-1} with
    h_{d+1,d} the positive-diagonal R factor of U~, so that the second
    sweep reproduces it exactly from the stored coefficients.
  * The sketched basis QR is updated one block column at a time by block
    classical Gram-Schmidt with one reorthogonalisation; the result is the
    R factor of S [U_d, U_{d+1}] (pinned against a fresh QR).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import scipy.linalg as sl

from .linalg import qr_pos, right_solve_upper, left_solve_upper, block_hessenberg
from .sketch import Sketch


@dataclasses.dataclass
class SideState:
    """One of the two Krylov recurrences (left: A, U; right: B^T, V)."""

    op: object            # sparse or dense operator applied as op @ X
    k: int
    S: Sketch
    r: int
    blocks: dict          # window (and all blocks when store_basis) {j: n x r}
    H: dict               # {(i, j): r x r}, 1-based Hessenberg blocks
    Q: np.ndarray         # s x (d+1) r sketched orthonormal basis
    T: np.ndarray         # (d+1) r x (d+1) r upper triangular
    first_R: np.ndarray   # ell: U_1 ell = C
    beta: np.ndarray      # R factor of S C = T_1 ell
    store_basis: bool


def _init_side(op, C, k, S, store_basis) -> SideState:
    """Algorithm 1's first step for one side: the skinny QR U_1 ell = C
    (positive diagonal), the QR of the sketch S U_1 = Q_1 T_1 (so T_1 is the
    R factor of S U_1, the reading taken above), and beta = T_1 ell, the R
    factor of S C that enters the projected right-hand side of Eq. (3.4)."""
    U1, ell = qr_pos(C)
    U1 = right_solve_upper(C, ell)  # U_1 = C ell^{-1}, reproducible in the replay
    Q1, T1 = qr_pos(S(U1))
    beta = T1 @ ell
    r = C.shape[1]
    return SideState(op, k, S, r, {1: U1}, {}, Q1, T1, ell, beta, store_basis)


def _arnoldi_step(st: SideState, d: int) -> None:
    """Truncated block Arnoldi step d (Algorithm 1) plus the sketch QR update."""
    r = st.r
    W = st.op @ st.blocks[d]                         # U~ = A U_d
    for i in range(max(1, d - st.k + 1), d + 1):     # MGS over the last k blocks
        h = st.blocks[i].T @ W
        W = W - st.blocks[i] @ h
        st.H[(i, d)] = h
    _, hn = qr_pos(W)                                # U_{d+1} h_{d+1,d} = U~
    st.H[(d + 1, d)] = hn
    st.blocks[d + 1] = right_solve_upper(W, hn)
    if not st.store_basis:
        for j in list(st.blocks):
            if j < d + 1 - st.k:
                del st.blocks[j]
    # QR update of S [U_d, U_{d+1}] (Proposition 2.1): new column block.
    w = st.S(st.blocks[d + 1])
    t1 = st.Q.T @ w
    w1 = w - st.Q @ t1
    t2 = st.Q.T @ w1
    w2 = w1 - st.Q @ t2
    qn, tau = qr_pos(w2)
    m = d * r
    T = np.zeros((m + r, m + r))
    T[:m, :m] = st.T
    T[:m, m:] = t1 + t2
    T[m:, m:] = tau
    st.T = T
    st.Q = np.hstack([st.Q, qn])


def projected_matrix(st: SideState, d: int):
    """H~_d = Hhat_d + Hhat E_d^T of Eqs. (2.9)-(2.10), formed directly.

    Hhat_d = T_d H_d T_d^{-1}, Hhat = T_H h_{d+1,d} tau_d^{-1}; returns
    (H~_d, hhat) with hhat = tau_{d+1} h_{d+1,d} tau_d^{-1}.
    """
    r = st.r
    m = d * r
    Hd = block_hessenberg(st.H, d, r)[:m, :m]
    Td = st.T[:m, :m]
    TH = st.T[:m, m:m + r]
    tau_d = st.T[m - r:m, m - r:m]
    tau_n = st.T[m:m + r, m:m + r]
    hn = st.H[(d + 1, d)]
    Hhat_d = right_solve_upper(Td @ Hd, Td)
    Hhat = right_solve_upper(TH @ hn, tau_d)
    Ht = Hhat_d.copy()
    Ht[:, m - r:] += Hhat
    hhat = right_solve_upper(tau_n @ hn, tau_d)
    return Ht, hhat


def bordering_update(Ht_d: np.ndarray, T_next: np.ndarray, H_col: np.ndarray,
                     h_sub: np.ndarray, h_diag: np.ndarray, r: int) -> np.ndarray:
    """Hhat_{d+1} = T_{d+1} H_{d+1} T_{d+1}^{-1} from H~_d (Section 5).

    Ht_d  : H~_d = Hhat_d + T_H h_{d+1,d} tau_d^{-1} E_d^T   (dr x dr)
    T_next: T_{d+1} = [[T_d, T_H], [0, tau_{d+1}]]             ((d+1)r square)
    H_col : [h_{1,d+1}; ...; h_{d,d+1}]                        (dr x r)
    h_sub : h_{d+1,d};  h_diag: h_{d+1,d+1}
    """
    m = Ht_d.shape[0]
    Td = T_next[:m, :m]
    TH = T_next[:m, m:]
    tau_n = T_next[m:, m:]
    tau_d = Td[m - r:, m - r:]
    out = np.zeros((m + r, m + r))
    out[:m, :m] = Ht_d
    tn_inv = lambda M: right_solve_upper(M, tau_n)
    out[:m, m:] = tn_inv(-Ht_d @ TH + Td @ H_col + TH @ h_diag)
    low = right_solve_upper(tau_n @ h_sub, tau_d)          # tau_{d+1} h tau_d^{-1}
    out[m:, m - r:m] = low
    out[m:, m:] = tn_inv(tau_n @ (-right_solve_upper(h_sub, tau_d) @ TH[m - r:, :] + h_diag))
    return out


def truncate(Y: np.ndarray, trunc_tol: float):
    """Y ~= Y1 Y2^T from the SVD, keeping sigma_i > trunc_tol * sigma_1."""
    P, sig, Qt = np.linalg.svd(Y)
    if sig.size == 0 or sig[0] == 0.0:
        return np.zeros((Y.shape[0], 0)), np.zeros((Y.shape[1], 0)), sig
    ell = int(np.sum(sig > trunc_tol * sig[0]))
    sq = np.sqrt(sig[:ell])
    return P[:, :ell] * sq[None, :], Qt[:ell, :].T * sq[None, :], sig


def replay(op, C: np.ndarray, ell: np.ndarray, H: dict, d: int, k: int, W: np.ndarray,
           r: int, stored: Optional[dict] = None):
    """Second Arnoldi sweep (Section 5): X = sum_j U_j W[j-th block rows].

    Regenerates U_1..U_d from the stored coefficients, without inner
    products, and accumulates the factor.  If `stored` holds the first-pass
    blocks they are compared on the way (returns the max abs difference).
    """
    X = np.zeros((C.shape[0], W.shape[1]))
    blocks = {1: right_solve_upper(C, ell)}
    maxdiff = 0.0
    for j in range(1, d + 1):
        if stored is not None:
            maxdiff = max(maxdiff, float(np.max(np.abs(blocks[j] - stored[j]))))
        X += blocks[j] @ W[(j - 1) * r:j * r, :]
        if j == d:
            break
        Wt = op @ blocks[j]
        for i in range(max(1, j - k + 1), j + 1):
            Wt = Wt - blocks[i] @ H[(i, j)]
        blocks[j + 1] = right_solve_upper(Wt, H[(j + 1, j)])
        for i in list(blocks):
            if i < j + 1 - k:
                del blocks[i]
    return X, maxdiff


def spkms(A, BT, C1, C2, *, k: int, s: int, tol: float, maxit: int, p: int = 1,
          seed: int = 0, sketch: str = "srht", k_right: Optional[int] = None,
          trunc_tol: float = 1e-12, same_sketch: bool = False,
          sketch_scale: Optional[float] = None, store_basis: bool = False,
          recover: bool = True, bordering: bool = False):
    """Run Algorithm 1.  Returns a dict with factors, history and internals.

    A: n1 x n1 and BT = B^T: n2 x n2 (anything supporting @), C1: n1 x r,
    C2: n2 x r.  k: truncation (window of k blocks), s: sketch rows,
    tol: relative tolerance on rho / ||beta1 beta2^T||_F, p: check period.
    sketch: 'srht' or 'identity'.  same_sketch: S_V = S_U (needs n1 = n2).
    bordering: also maintain H~ by the Section 5 update (returned for pins).
    """
    C1 = np.asarray(C1, dtype=np.float64)
    C2 = np.asarray(C2, dtype=np.float64)
    if C1.ndim == 1:
        C1 = C1[:, None]
    if C2.ndim == 1:
        C2 = C2[:, None]
    n1, r = C1.shape
    n2 = C2.shape[0]
    SU = Sketch(n1, s, seed, 0, sketch, sketch_scale)
    SV = Sketch(n2, s, seed, 0 if same_sketch else 1, sketch, sketch_scale)
    U = _init_side(A, C1, k, SU, store_basis)
    V = _init_side(BT, C2, k if k_right is None else k_right, SV, store_basis)
    F11 = U.beta @ V.beta.T
    nrm_rhs = np.linalg.norm(F11)
    hist = []
    Y = None
    Ht = Gt = None
    bord = {"U": None, "V": None, "checks": []}
    d = 0
    converged = False
    for d in range(1, maxit + 1):
        _arnoldi_step(U, d)
        _arnoldi_step(V, d)
        if bordering:
            for key, st in (("U", U), ("V", V)):
                if d == 1:
                    bord[key] = None
                else:
                    prev = bord[key]
                    bord[key] = bordering_update(
                        prev, st.T[:d * r, :d * r],
                        block_hessenberg(st.H, d, r)[:(d - 1) * r, (d - 1) * r:d * r],
                        st.H[(d, d - 1)], st.H[(d, d)], r)
            # keep H~_d (with the E_d^T correction) for the next update
            for key, st in (("U", U), ("V", V)):
                Htd, _ = projected_matrix(st, d)
                if bord[key] is not None:
                    m = d * r
                    Hhat_only = bord[key].copy()
                    TH = st.T[:m, m:m + r]
                    tau_d = st.T[m - r:m, m - r:m]
                    Hhat_only[:, m - r:] += right_solve_upper(TH @ st.H[(d + 1, d)], tau_d)
                    bord["checks"].append((key, d, float(np.max(np.abs(Hhat_only - Htd))),
                                           float(np.max(np.abs(Htd)))))
                bord[key] = Htd
        if d % p == 0 or d == maxit:
            m = d * r
            Ht, hhat = projected_matrix(U, d)
            Gt, ghat = projected_matrix(V, d)
            F = np.zeros((m, m))
            F[:r, :r] = F11
            Y = sl.solve_sylvester(Ht, Gt.T, F)            # Eq. (3.4)
            rho = np.sqrt(np.linalg.norm(hhat @ Y[m - r:, :]) ** 2
                          + np.linalg.norm(Y[:, m - r:] @ ghat.T) ** 2)   # Eq. (3.5)
            hist.append((d, rho, rho / nrm_rhs))
            if rho / nrm_rhs < tol:
                converged = True
                break
    out = dict(d=d, r=r, converged=converged, hist=hist, Y=Y, Ht=Ht, Gt=Gt,
               T_U=U.T, T_V=V.T, H=U.H, G=V.H, Q_U=U.Q, Q_V=V.Q,
               beta1=U.beta, beta2=V.beta, ell1=U.first_R, ell2=V.first_R,
               SU=SU, SV=SV, rho=hist[-1][1] if hist else None,
               rel_rho=hist[-1][2] if hist else None, bordering=bord)
    if store_basis:
        out["U_blocks"] = U.blocks
        out["V_blocks"] = V.blocks
    if recover and Y is not None:
        m = d * r
        Y1, Y2, sig = truncate(Y, trunc_tol)
        W1 = left_solve_upper(U.T[:m, :m], Y1)
        W2 = left_solve_upper(V.T[:m, :m], Y2)
        X1, diffU = replay(A, C1, U.first_R, U.H, d, U.k, W1, r,
                           U.blocks if store_basis else None)
        X2, diffV = replay(BT, C2, V.first_R, V.H, d, V.k, W2, r,
                           V.blocks if store_basis else None)
        out.update(X1=X1, X2=X2, rank=Y1.shape[1], sigma=sig, W1=W1, W2=W2,
                   replay_maxdiff=max(diffU, diffV))
    return out


def dense_solution(res: dict) -> np.ndarray:
    """X_d = U_d T_U^{-1} Y T_V^{-T} V_d^T from a run with store_basis=True."""
    d, r = res["d"], res["r"]
    m = d * r
    Ud = np.hstack([res["U_blocks"][j] for j in range(1, d + 1)])
    Vd = np.hstack([res["V_blocks"][j] for j in range(1, d + 1)])
    L = right_solve_upper(Ud, res["T_U"][:m, :m])
    R = right_solve_upper(Vd, res["T_V"][:m, :m])
    return L @ res["Y"] @ R.T
