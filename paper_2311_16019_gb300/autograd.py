"""Differentiating through the sketched solver: a torch.autograd.Function for
the bilinear loss L = u^T X v of the solution of

    A(theta) X + X B(theta) = C1 C2^T,   A(theta) = A0 + theta A_theta,
                                         B(theta) = B0 + theta B_theta.

Differentiating Eq. (1.1) gives A dX + dX B = dC - dA X - X dB, so with the
adjoint Lambda solving A^T Lambda + Lambda B^T = u v^T (the same solver on
the operators A^T and B, right-hand side of rank one):

    dL/dC1 = Lambda C2,   dL/dC2 = Lambda^T C1,
    dL/dtheta = -<Lambda, A_theta X + X B_theta>_F,
    dL/du = X v,          dL/dv = X^T u.

Both solves and the C1, C2 and theta gradients run in libspk (spk_solve,
spk_solve_adjoint, spk_adjoint_gradients).  This module assembles A(theta),
B(theta) on the host, and evaluates the loss itself and its u, v gradients
(products of the n x l factors with one vector) with torch.
"""
from __future__ import annotations

import dataclasses
import scipy.sparse as sp

from . import spk


@dataclasses.dataclass
class OperatorFamily:
    """A(theta) = A0 + theta A_theta and B(theta) = B0 + theta B_theta (CSR)."""

    A0: sp.csr_matrix
    A_theta: sp.csr_matrix
    B0: sp.csr_matrix
    B_theta: sp.csr_matrix

    @classmethod
    def from_problem(cls, P) -> "OperatorFamily":
        """Split a problem's operators at its own theta into the two parts."""
        return cls(sp.csr_matrix(P.A - P.theta * P.A_theta), sp.csr_matrix(P.A_theta),
                   sp.csr_matrix(P.B - P.theta * P.B_theta), sp.csr_matrix(P.B_theta))

    def at(self, theta: float):
        A = sp.csr_matrix(self.A0 + theta * self.A_theta)
        B = sp.csr_matrix(self.B0 + theta * self.B_theta)
        A.sort_indices()
        B.sort_indices()
        return A, B


def _torch():
    import torch
    return torch


class _Bilinear:
    """Holder for the autograd.Function (built lazily so that importing this
    module does not import torch)."""

    fn = None


def _make_function():
    torch = _torch()

    class SylvesterBilinear(torch.autograd.Function):
        @staticmethod
        def forward(ctx, C1, C2, theta, u, v, family: OperatorFamily, opts: dict):
            th = float(theta.detach().cpu())
            A, B = family.at(th)
            sol = spk.solve(A, sp.csr_matrix(B.T), C1.detach(), C2.detach(), **opts)
            X1, X2 = sol.X1, sol.X2
            uu, vv = u.detach().reshape(-1), v.detach().reshape(-1)
            if X1 is None:
                val = torch.zeros((), dtype=torch.float64, device=C1.device)
            else:
                val = (uu @ X1) @ (X2.T @ vv)
            ctx.family, ctx.opts, ctx.A, ctx.B = family, opts, A, B
            ctx.sol = sol
            ctx.save_for_backward(C1, C2, u, v)
            return val

        @staticmethod
        def backward(ctx, gL):
            C1, C2, u, v = ctx.saved_tensors
            uu, vv = u.detach().reshape(-1, 1), v.detach().reshape(-1, 1)
            lam = spk.solve_adjoint(sp.csr_matrix(ctx.A.T), ctx.B, uu, vv, **ctx.opts)
            dC1, dC2, dth = spk.adjoint_gradients(spk.result_view(ctx.sol), spk.result_view(lam),
                                                  C1.detach(), C2.detach(), ctx.family.A_theta,
                                                  ctx.family.B_theta)
            X1, X2 = ctx.sol.X1, ctx.sol.X2
            g = gL.to(torch.float64)
            du = (X1 @ (X2.T @ vv.reshape(-1))).reshape(u.shape) if X1 is not None else None
            dv = (X2 @ (X1.T @ uu.reshape(-1))).reshape(v.shape) if X1 is not None else None
            dtheta = torch.tensor(dth, dtype=torch.float64, device=C1.device)
            return (g * dC1.reshape(C1.shape), g * dC2.reshape(C2.shape), g * dtheta,
                    None if du is None else g * du, None if dv is None else g * dv, None, None)

    return SylvesterBilinear


def bilinear_loss(C1, C2, theta, u, v, family: OperatorFamily, **opts):
    """L = u^T X v for A(theta) X + X B(theta) = C1 C2^T (differentiable in C1,
    C2, theta, u and v; tensors on the GPU, float64)."""
    if _Bilinear.fn is None:
        _Bilinear.fn = _make_function()
    return _Bilinear.fn.apply(C1, C2, theta, u, v, family, opts)
