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
spk_solve_adjoint, spk_adjoint_gradients).  The operators A(theta),
B(theta)^T, A(theta)^T and B(theta) live on the device on the union sparsity
pattern of their two parts, set up once per family; their values
v0 + theta v_theta are formed by libspk's FP64 product (spk_dense_gemm) at
each theta.  The loss itself and its u, v gradients (products of the n x l
factors with one vector) are torch operations.
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
        """A(theta), B(theta) on the host (for checks against the oracle)."""
        A = sp.csr_matrix(self.A0 + theta * self.A_theta)
        B = sp.csr_matrix(self.B0 + theta * self.B_theta)
        A.sort_indices()
        B.sort_indices()
        return A, B

    def device_ops(self, theta, device: int = 0):
        """A(theta), B(theta)^T, A(theta)^T, B(theta) as device CSR matrices;
        `theta` is a device scalar tensor."""
        torch = _torch()
        dev = _family_device(self, device)
        coef = torch.cat([torch.ones(1, dtype=torch.float64, device=theta.device),
                          theta.detach().reshape(1).to(torch.float64)])
        out = []
        for name in ("A", "BT", "AT", "B"):
            op = dev[name]
            nnz = op.val.numel()
            # values = [v0, v_theta] [1, theta]^T on the union pattern
            spk.dense_gemm_device(nnz, 1, 2, op.parts, nnz, coef, 2, op.val, nnz, device=device)
            out.append(op.csr)
        return tuple(out)

    def device_theta_ops(self, device: int = 0):
        """A_theta and B_theta as device CSR matrices (for the theta gradient)."""
        dev = _family_device(self, device)
        return dev["A_theta"], dev["B_theta"]


def union_pattern(X0, Xt):
    """The union of the sparsity patterns of X0 and Xt (CSR, sorted) and the
    two matrices' values on it: (shape, indptr, indices, v0, vt), so that
    X0 + theta Xt has the values v0 + theta vt on that pattern."""
    import numpy as np
    X0, Xt = sp.csr_matrix(X0), sp.csr_matrix(Xt)
    P = sp.csr_matrix(abs(X0) + abs(Xt))
    P.eliminate_zeros()
    P.sort_indices()
    rows, cols = P.nonzero()
    v0 = np.asarray(X0[rows, cols], dtype=np.float64).ravel()
    vt = np.asarray(Xt[rows, cols], dtype=np.float64).ravel()
    return P.shape, P.indptr.astype(np.int32), P.indices.astype(np.int32), v0, vt


class _DeviceOperator:
    """X0 + theta X_theta on the union of the two sparsity patterns: the
    pattern (int32) and the two value arrays on the device, and the values at
    the last theta."""

    def __init__(self, X0, Xt, device):
        import numpy as np
        torch = _torch()
        shape, indptr, indices, v0, vt = union_pattern(X0, Xt)
        dv = "cuda:%d" % device
        self.rowptr = torch.as_tensor(indptr, device=dv)
        self.col = torch.as_tensor(indices, device=dv)
        # column-major nnz x 2: [v0, v_theta]
        self.parts = torch.as_tensor(np.stack([v0, vt]), device=dv).contiguous()
        self.val = torch.empty(len(v0), dtype=torch.float64, device=dv)
        self.csr = spk.DeviceCSR.from_device(shape, self.rowptr, self.col, self.val)


def _family_device(fam: "OperatorFamily", device: int):
    cache = fam.__dict__.setdefault("_device_cache", {})
    if device not in cache:
        cache[device] = {
            "A": _DeviceOperator(fam.A0, fam.A_theta, device),
            "BT": _DeviceOperator(fam.B0.T, fam.B_theta.T, device),
            "AT": _DeviceOperator(fam.A0.T, fam.A_theta.T, device),
            "B": _DeviceOperator(fam.B0, fam.B_theta, device),
            "A_theta": spk.DeviceCSR(fam.A_theta),
            "B_theta": spk.DeviceCSR(fam.B_theta),
        }
    return cache[device]


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
            dA, dBT, dAT, dB = family.device_ops(theta)
            sol = spk.solve(dA, dBT, C1.detach(), C2.detach(), **opts)
            X1, X2 = sol.X1, sol.X2
            uu, vv = u.detach().reshape(-1), v.detach().reshape(-1)
            if X1 is None:
                val = torch.zeros((), dtype=torch.float64, device=C1.device)
            else:
                val = (uu @ X1) @ (X2.T @ vv)
            ctx.family, ctx.opts, ctx.AT, ctx.B = family, opts, dAT, dB
            ctx.sol = sol
            ctx.save_for_backward(C1, C2, u, v)
            return val

        @staticmethod
        def backward(ctx, gL):
            C1, C2, u, v = ctx.saved_tensors
            uu, vv = u.detach().reshape(-1, 1), v.detach().reshape(-1, 1)
            lam = spk.solve_adjoint(ctx.AT, ctx.B, uu, vv, **ctx.opts)
            dAth, dBth = ctx.family.device_theta_ops()
            dC1, dC2, dth = spk.adjoint_gradients(spk.result_view(ctx.sol), spk.result_view(lam),
                                                  C1.detach(), C2.detach(), dAth, dBth)
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
