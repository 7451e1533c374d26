"""Seeded synthetic inputs for AX + XB = C1 C2^T (the problem of Eq. (1.1)).

This module is shared by the CUDA path, the CPU oracle, the tests and the
benchmark.  It holds NONE of the solver's arithmetic: it only builds the
problem data -- sparse coefficient matrices in CSR form, their transposes,
and Gaussian right-hand-side factors -- from a seed.

Operators (the convection-diffusion family of Section 6, Examples 6.1/6.3,
re-specified for the synthetic workloads):
  * unit square / cube, N interior nodes per direction, h = 1/(N+1),
    lexicographic ordering with x fastest (index = i + N*j [+ N*N*l]);
  * -Laplacian by the (1/h^2)-scaled 5-point (2-D) or 7-point (3-D) stencil
    with homogeneous Dirichlet boundary values;
  * convection w . grad u by first-order upwinding: at a node where w_x > 0
    the backward difference (u_i - u_{i-1})/h is used, where w_x < 0 the
    forward difference (u_{i+1} - u_i)/h, and likewise in y and z;
  * A = -Lap + theta * (w_A . grad),  B = -Lap + theta * (w_B . grad).
Upwinding keeps the 5/7-point pattern, so nnz = 5N^2 - 4N (2-D) and
7N^3 - 6N^2 (3-D).

The right space of the method is K(B^T, C2) (Eq. (1.2)); every problem
therefore carries B^T in CSR form as well as B.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional, Tuple

import numpy as np
import scipy.sparse as sp

__all__ = [
    "Problem",
    "laplacian",
    "convdiff_2d",
    "convdiff_3d",
    "rhs_factors",
    "diagonal_problem",
    "workload",
    "WORKLOADS",
    "batched_instances",
]


@dataclasses.dataclass
class Problem:
    """One Sylvester problem A X + X B = C1 C2^T with CSR operators.

    A, B, BT, AT are scipy.sparse.csr_matrix (float64, int32 indices, sorted
    columns).  A_theta / B_theta are the convection parts (dA/dtheta,
    dB/dtheta) when the operator family has a convection coefficient.
    """

    name: str
    A: sp.csr_matrix
    B: sp.csr_matrix
    C1: np.ndarray
    C2: np.ndarray
    theta: float = 0.0
    A_theta: Optional[sp.csr_matrix] = None
    B_theta: Optional[sp.csr_matrix] = None
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def AT(self) -> sp.csr_matrix:
        return _csr(self.A.T)

    @property
    def BT(self) -> sp.csr_matrix:
        return _csr(self.B.T)

    @property
    def n1(self) -> int:
        return self.A.shape[0]

    @property
    def n2(self) -> int:
        return self.B.shape[0]

    @property
    def r(self) -> int:
        return self.C1.shape[1]


def _csr(M) -> sp.csr_matrix:
    M = sp.csr_matrix(M, dtype=np.float64)
    M.sum_duplicates()
    M.sort_indices()
    M.indptr = M.indptr.astype(np.int32)
    M.indices = M.indices.astype(np.int32)
    return M


def _second_diff(N: int, h: float) -> sp.csr_matrix:
    e = np.ones(N)
    return sp.diags([-e[:-1], 2.0 * e, -e[:-1]], [-1, 0, 1], format="csr") / (h * h)


def _backward(N: int, h: float) -> sp.csr_matrix:
    e = np.ones(N)
    return sp.diags([-e[:-1], e], [-1, 0], format="csr") / h


def _forward(N: int, h: float) -> sp.csr_matrix:
    e = np.ones(N)
    return sp.diags([-e, e[:-1]], [0, 1], format="csr") / h


def _kron_axis(mats, axis: int, dim: int, N: int):
    """I x ... x M x ... x I with M acting on `axis` (0 = x, fastest)."""
    I = sp.identity(N, format="csr")
    out = None
    # lexicographic x fastest: kron(..., I_y, M_x) -> the last factor is x.
    for ax in reversed(range(dim)):
        f = mats if ax == axis else I
        out = f if out is None else sp.kron(out, f, format="csr")
    return out


def laplacian(N: int, dim: int = 2) -> sp.csr_matrix:
    """-Delta_h on N^dim interior nodes (Dirichlet), scaled by 1/h^2."""
    h = 1.0 / (N + 1)
    T = _second_diff(N, h)
    L = None
    for ax in range(dim):
        term = _kron_axis(T, ax, dim, N)
        L = term if L is None else L + term
    return _csr(L)


def _grid(N: int, dim: int):
    h = 1.0 / (N + 1)
    x = np.arange(1, N + 1) * h
    grids = np.meshgrid(*([x] * dim), indexing="ij")
    # grids[a] indexed [i_x, i_y, (i_z)]; flatten with x fastest.
    return [g.transpose(tuple(reversed(range(dim)))).ravel() for g in grids]


def _upwind(N: int, dim: int, wind: Callable) -> sp.csr_matrix:
    h = 1.0 / (N + 1)
    coords = _grid(N, dim)
    w = wind(*coords)
    C = None
    for ax in range(dim):
        wa = np.broadcast_to(np.asarray(w[ax], dtype=np.float64), coords[0].shape)
        Db = _kron_axis(_backward(N, h), ax, dim, N)
        Df = _kron_axis(_forward(N, h), ax, dim, N)
        term = sp.diags(np.maximum(wa, 0.0)) @ Db + sp.diags(np.minimum(wa, 0.0)) @ Df
        C = term if C is None else C + term
    return _csr(C)


def convdiff_2d(N: int, theta: float, wind: Callable):
    """(A, dA/dtheta) for A = -Lap_h + theta * (w . grad) on the unit square."""
    L = laplacian(N, 2)
    C = _upwind(N, 2, wind)
    return _csr(L + theta * C), C


def convdiff_3d(N: int, theta: float, wind: Callable):
    """(A, dA/dtheta) for A = -Lap_h + theta * (w . grad) on the unit cube."""
    L = laplacian(N, 3)
    C = _upwind(N, 3, wind)
    return _csr(L + theta * C), C


def rhs_factors(n1: int, n2: int, r: int, seed: int) -> Tuple[np.ndarray, np.ndarray]:
    """C1 (n1 x r), C2 (n2 x r) with i.i.d. N(0,1) entries from one seed."""
    rng = np.random.default_rng(seed)
    C1 = rng.standard_normal((n1, r))
    C2 = rng.standard_normal((n2, r))
    return C1, C2


def diagonal_problem(n: int, distinct: int, r: int, seed: int) -> Problem:
    """Diagonal A, B with `distinct` distinct positive values each.

    X_ij = (C1 C2^T)_ij / (a_i + b_j) in closed form, and the block Krylov
    spaces reach their full dimension distinct*r after `distinct` steps.
    """
    rng = np.random.default_rng(seed)
    av = np.linspace(1.0, 4.0, distinct)
    bv = np.linspace(0.5, 3.0, distinct)
    a = np.repeat(av, n // distinct + 1)[:n]
    b = np.repeat(bv, n // distinct + 1)[:n]
    a = a[rng.permutation(n)]
    b = b[rng.permutation(n)]
    C1, C2 = rhs_factors(n, n, r, seed + 1000)
    return Problem("diagonal", _csr(sp.diags(a)), _csr(sp.diags(b)), C1, C2,
                   meta={"a": a, "b": b})


def _wind_c2_A(x, y):
    return (x, y)


def _wind_c2_B(x, y):
    return (y, -x)


def _wind_c3_A(x, y, z):
    return (1.0, 1.0, 1.0)


def _wind_c3_B(x, y, z):
    return (1.0, -1.0, 0.0)


def _central(N: int, h: float) -> sp.csr_matrix:
    e = np.ones(N)
    return sp.diags([-e[:-1], e[:-1]], [-1, 1], format="csr") / (2.0 * h)


def centered_convdiff(N: int, dim: int, nu: float, wind: Callable) -> sp.csr_matrix:
    """-nu Lap_h + w . grad_h with centred differences for both terms
    (the operators of the paper's Examples 6.1 and 6.3): N^dim interior
    nodes of the unit square or cube, h = 1/(N+1), Dirichlet, x fastest."""
    h = 1.0 / (N + 1)
    coords = _grid(N, dim)
    w = wind(*coords)
    A = nu * laplacian(N, dim)
    for ax in range(dim):
        wa = np.broadcast_to(np.asarray(w[ax], dtype=np.float64), coords[0].shape)
        A = A + sp.diags(wa) @ _kron_axis(_central(N, h), ax, dim, N)
    return _csr(A)


def _wind_ex61_A(x, y):
    return (1.0, 1.0)


def _wind_ex61_B(x, y):
    return (3.0 * y * (1.0 - x * x), -2.0 * x * (1.0 - y * y))


def _wind_ex63_A(x, y, z):
    return (x * np.sin(x), y * np.cos(y), np.exp(z * z - 1.0))


def _wind_ex63_B(x, y, z):
    return ((1.0 - x * x) * y * z, 1.0, np.exp(z))


def _unit_rhs(n1, n2, r, seed):
    """N(0,1) factors scaled so that ||C1 C2^T||_F = 1 (as in the paper's
    examples)."""
    C1, C2 = rhs_factors(n1, n2, r, seed)
    _, R1 = np.linalg.qr(C1)
    _, R2 = np.linalg.qr(C2)
    nrm = np.linalg.norm(R1 @ R2.T)
    return C1 / np.sqrt(nrm), C2 / np.sqrt(nrm)


def _conv2d_problem(name, N, theta, r, seed) -> Problem:
    A, CA = convdiff_2d(N, theta, _wind_c2_A)
    B, CB = convdiff_2d(N, theta, _wind_c2_B)
    C1, C2 = rhs_factors(A.shape[0], B.shape[0], r, seed)
    return Problem(name, A, B, C1, C2, theta=theta, A_theta=CA, B_theta=CB,
                   meta={"N": N, "dim": 2})


def workload(name: str) -> Problem:
    """The named synthetic workloads (sizes and seeds fixed here).

    lap32_r1      : A = B = -Lap_h, 32x32 grid (n=1024), r=1, seed 0
    cd2d_512_r4   : 2-D conv-diff 512x512 (n=262144), theta=10, r=4, seed 1
    cd3d_96_r2    : 3-D conv-diff 96^3 (n=884736), theta=20, r=2, seed 2
    cd2d_256_r2   : 2-D conv-diff 256x256 (n=65536), theta=10, r=2, seed 3
    small variants for fast tests: lap16_r1, cd2d_32_r2, cd2d_64_r4, cd3d_16_r2
    ex61_<N>_nu<nu>_r<r> : Example 6.1 (centred FD, nu, w_A = (1,1),
                           w_B = (3y(1-x^2), -2x(1-y^2))), ||C1 C2^T||_F = 1
    ex63_<N>             : Example 6.3 (3-D centred FD, nu = 0.005), r = 1
    """
    if name.startswith("lap"):
        N = int(name[3:].split("_")[0])
        r = int(name.split("_r")[1])
        L = laplacian(N, 2)
        C1, C2 = rhs_factors(L.shape[0], L.shape[0], r, 0)
        return Problem(name, L, L.copy(), C1, C2, meta={"N": N, "dim": 2})
    if name.startswith("cd2d_"):
        N = int(name.split("_")[1])
        r = int(name.split("_r")[1])
        seed = {512: 1, 256: 3}.get(N, 7)
        return _conv2d_problem(name, N, 10.0, r, seed)
    if name.startswith("ex61_"):
        # ex61_<N>_nu<nu>_r<r>: Example 6.1's 2-D operators, N^2 nodes
        parts = name.split("_")
        N = int(parts[1])
        nu = float(parts[2][2:])
        r = int(parts[3][1:])
        A = centered_convdiff(N, 2, nu, _wind_ex61_A)
        B = centered_convdiff(N, 2, nu, _wind_ex61_B)
        C1, C2 = _unit_rhs(A.shape[0], B.shape[0], r, 61)
        return Problem(name, A, B, C1, C2, meta={"N": N, "dim": 2, "nu": nu})
    if name.startswith("ex63_"):
        # ex63_<N>: Example 6.3's 3-D operators (nu = 0.005), N^3 nodes, r = 1
        N = int(name.split("_")[1])
        A = centered_convdiff(N, 3, 0.005, _wind_ex63_A)
        B = centered_convdiff(N, 3, 0.005, _wind_ex63_B)
        C1, C2 = _unit_rhs(A.shape[0], B.shape[0], 1, 63)
        return Problem(name, A, B, C1, C2, meta={"N": N, "dim": 3, "nu": 0.005})
    if name.startswith("cd3d_"):
        N = int(name.split("_")[1])
        r = int(name.split("_r")[1])
        A, CA = convdiff_3d(N, 20.0, _wind_c3_A)
        B, CB = convdiff_3d(N, 20.0, _wind_c3_B)
        C1, C2 = rhs_factors(A.shape[0], B.shape[0], r, 2 if N == 96 else 8)
        return Problem(name, A, B, C1, C2, theta=20.0, A_theta=CA, B_theta=CB,
                       meta={"N": N, "dim": 3})
    raise KeyError(name)


WORKLOADS = {
    # name: (default solver options used by tests/bench for that workload)
    "lap32_r1": dict(k=2, s=600, maxit=300, p=1, tol=1e-8),
    "cd2d_512_r4": dict(k=4, s=12000, maxit=1500, p=20, tol=1e-8),
    "cd3d_96_r2": dict(k=3, s=3200, maxit=800, p=20, tol=1e-8),
    "cd2d_256_r2": dict(k=4, s=6000, maxit=1500, p=20, tol=1e-8),
}


def batched_instances(count: int = 64, seed: int = 4, nmin: int = 64, nmax: int = 384):
    """The uneven batch: N ~ U{nmin..nmax}, theta ~ U[1,50], r ~ U{1,2,4}."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(rng.integers(nmin, nmax + 1))
        theta = float(rng.uniform(1.0, 50.0))
        r = int(rng.choice([1, 2, 4]))
        p = _conv2d_problem(f"batch{i}", N, theta, r, seed * 100000 + i)
        out.append(p)
    return out
