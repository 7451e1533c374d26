"""Dense FP64 gradient of L = u^T X v for A X + X B = C1 C2^T (test infrastructure).

With A = L_A + theta A_theta and B = L_B + theta B_theta, the adjoint
Lambda solves A^T Lambda + Lambda B^T = u v^T and
    dL/dC1 = Lambda C2,  dL/dC2 = Lambda^T C1,
    dL/dtheta = -<Lambda, A_theta X + X B_theta>_F.
(Differentiate A X + X B = C: A dX + dX B = dC - dA X - X dB, then
<u v^T, dX> = <Lambda, dC - dA X - X dB>.)  Dense: small n only.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl


def dense_solve(A, B, C1, C2):
    """X of Eq. (1.1), densely, by SciPy's Bartels-Stewart routine (the
    method of the lyap solver the paper's experiments use for the projected
    equations, Section 6).  Small n only."""
    A = np.asarray(A.todense() if hasattr(A, "todense") else A)
    B = np.asarray(B.todense() if hasattr(B, "todense") else B)
    return sl.solve_sylvester(A, B, C1 @ C2.T)


def dense_gradient(A, B, A_theta, B_theta, C1, C2, u, v):
    """L = u^T X v and its gradients by the formulas of this module's
    docstring: Lambda from the transposed equation of Eq. (1.1),
    A^T Lambda + Lambda B^T = u v^T, then dL/dC1 = Lambda C2,
    dL/dC2 = Lambda^T C1, dL/dtheta = -<Lambda, A_theta X + X B_theta>_F.
    The paper has no adjoint; this differentiates its Eq. (1.1) directly."""
    A = np.asarray(A.todense() if hasattr(A, "todense") else A)
    B = np.asarray(B.todense() if hasattr(B, "todense") else B)
    At = np.asarray(A_theta.todense() if hasattr(A_theta, "todense") else A_theta)
    Bt = np.asarray(B_theta.todense() if hasattr(B_theta, "todense") else B_theta)
    X = sl.solve_sylvester(A, B, C1 @ C2.T)
    Lam = sl.solve_sylvester(A.T, B.T, np.outer(u, v))
    L = float(u @ X @ v)
    return dict(L=L, X=X, Lam=Lam, dC1=Lam @ C2, dC2=Lam.T @ C1,
                dtheta=-float(np.sum(Lam * (At @ X + X @ Bt))),
                du=X @ v, dv=X.T @ u)
