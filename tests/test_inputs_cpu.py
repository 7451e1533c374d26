"""Pins of the seeded input generators (the synthetic convection-diffusion
operators of Section 6 and the low-rank right-hand sides of Eq. (1.1)).

Both the CUDA path and the oracle take their problems from
paper_2311_16019_gb300/inputs.py, so a mistake there would pass every parity
test.  These CPU tests pin the generators to facts that do not depend on the
code: stencil sizes, the closed-form spectrum of the discrete Laplacian,
exactness of the difference quotients on low-degree polynomials, the sign
pattern of upwinding, skew-symmetry of centred convection, and the stated
distributions of the batched sweep.
"""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2311_16019_gb300 import inputs as I


def _grid(N, dim):
    h = 1.0 / (N + 1)
    x = np.arange(1, N + 1) * h
    g = np.meshgrid(*([x] * dim), indexing="ij")
    # x fastest: index = i + N j (+ N^2 l)
    return [a.transpose(tuple(reversed(range(dim)))).ravel() for a in g], h


def _interior(coords, h):
    """Nodes whose neighbours in every direction are grid nodes, so that no
    difference quotient there meets a Dirichlet value."""
    m = np.ones(coords[0].shape, dtype=bool)
    for c in coords:
        m &= (c > 1.5 * h) & (c < 1.0 - 1.5 * h)
    return m


@pytest.mark.parametrize("name,nnz,n", [
    ("lap32_r1", 5 * 32 ** 2 - 4 * 32, 32 ** 2),
    ("cd2d_256_r2", 5 * 256 ** 2 - 4 * 256, 256 ** 2),
    ("cd2d_512_r4", 5 * 512 ** 2 - 4 * 512, 512 ** 2),
    ("cd3d_16_r2", 7 * 16 ** 3 - 6 * 16 ** 2, 16 ** 3),
    ("cd3d_96_r2", 7 * 96 ** 3 - 6 * 96 ** 2, 96 ** 3),
])
def test_stencil_sizes(name, nnz, n):
    """5-point (2-D) and 7-point (3-D) patterns: every interior node couples to
    its neighbours, minus the ones cut off by the Dirichlet boundary."""
    P = I.workload(name)
    assert P.n1 == P.n2 == n
    for M in (P.A, P.B, P.BT):
        assert M.nnz == nnz
        assert M.indptr.dtype == np.int32 and M.indices.dtype == np.int32
        assert M.has_sorted_indices
    assert abs(P.BT - P.B.T).max() == 0.0
    assert P.C1.shape == (n, P.r) and P.C2.shape == (n, P.r)


@pytest.mark.parametrize("N,dim", [(6, 2), (4, 3)])
def test_laplacian_spectrum_closed_form(N, dim):
    """Eigenvalues of -Lap_h with Dirichlet values: sums over the axes of
    (4/h^2) sin^2(j pi h / 2), j = 1..N."""
    h = 1.0 / (N + 1)
    lam1 = 4.0 / h ** 2 * np.sin(np.arange(1, N + 1) * np.pi * h / 2) ** 2
    lam = lam1
    for _ in range(dim - 1):
        lam = (lam[:, None] + lam1[None, :]).ravel()
    ev = np.linalg.eigvalsh(I.laplacian(N, dim).toarray())
    assert np.allclose(np.sort(ev), np.sort(lam), rtol=1e-12, atol=0)


@pytest.mark.parametrize("dim", [2, 3])
def test_laplacian_exact_on_quadratic(dim):
    """The 3-point second difference is exact on quadratics.  f = prod_a
    q(x_a) with q(t) = t(1-t) is zero on the whole boundary, so at every node
    -Lap_h f = sum_a 2 prod_{b != a} q(x_b) exactly."""
    N = 9
    coords, h = _grid(N, dim)
    q = [c * (1.0 - c) for c in coords]
    f = np.prod(q, axis=0)
    want = sum(2.0 * np.prod([q[b] for b in range(dim) if b != a], axis=0)
               for a in range(dim))
    assert np.allclose(I.laplacian(N, dim) @ f, want, rtol=1e-12, atol=1e-13)


def test_upwind_2d_axes_and_directions():
    """Upwinding of Section 6's convection term, x fastest in the ordering.
    Difference quotients are exact on linear functions at nodes away from
    the boundary, so w . grad_h f = w . grad f there, whichever side each
    one-sided quotient takes.  A swapped axis order would exchange the two
    wind components and fail; so would a downwind quotient at the nodes
    next to the boundary (checked on f = x, whose Dirichlet value at x = 0
    is the true one)."""
    N = 12
    theta = 10.0
    (x, y), h = _grid(N, 2)
    A, CA = I.convdiff_2d(N, theta, lambda x, y: (x, y))
    B, CB = I.convdiff_2d(N, theta, lambda x, y: (y, -x))
    m = _interior([x, y], h)
    f = x + 3.0 * y
    assert np.allclose((CA @ f)[m], (x + 3.0 * y)[m], rtol=1e-12)
    assert np.allclose((CB @ f)[m], (y - 3.0 * x)[m], rtol=1e-12)
    # wind (x, y) > 0: backward in x, so the x = 0 side sees f(0) = 0 = x
    # exactly; a forward quotient would fail on the x = 1 - h column
    edge = (y > 1.5 * h) & (y < 1.0 - 1.5 * h)
    assert np.allclose((CA @ x)[edge], x[edge], rtol=1e-12)
    # wind_x of B is y > 0 (backward), wind_y is -x < 0 (forward): on f = y
    # the forward quotient meets y = 1 - h's Dirichlet neighbour 0
    top = (y > 1.0 - 1.5 * h) & (x > 1.5 * h) & (x < 1.0 - 1.5 * h)
    assert np.allclose((CB @ y)[top], (-x * (0.0 - y) / h)[top], rtol=1e-12)
    # A = -Lap_h + theta * C exactly
    assert abs(A - I.laplacian(N, 2) - theta * CA).max() < 1e-9


@pytest.mark.parametrize("name", ["cd2d_32_r2", "cd3d_16_r2"])
def test_upwind_operators_are_m_matrices(name):
    """First-order upwinding keeps a positive diagonal, non-positive
    off-diagonal entries and non-negative row sums (weak diagonal dominance)."""
    P = I.workload(name)
    for M in (P.A, P.B):
        D = M.diagonal()
        off = M - sp.diags(D)
        assert (D > 0).all()
        assert off.data.max() <= 0.0
        assert (np.asarray(M.sum(axis=1)).ravel() >= -1e-9 * D).all()
    # and the convection part is linear in theta
    L = I.laplacian(P.meta["N"], P.meta["dim"])
    assert abs(P.A - L - P.theta * P.A_theta).max() < 1e-8 * abs(P.A).max()
    assert abs(P.B - L - P.theta * P.B_theta).max() < 1e-8 * abs(P.B).max()


def test_upwind_3d_constant_winds():
    """Winds 20 (1,1,1) for A and 20 (1,-1,0) for B: on f = x + 2y + 3z the
    backward/forward quotients give w . grad f exactly (away from the sides
    where a forward difference meets the Dirichlet value)."""
    P = I.workload("cd3d_16_r2")
    N = 16
    (x, y, z), h = _grid(N, 3)
    f = x + 2 * y + 3 * z
    m = _interior([x, y, z], h)
    assert np.allclose((P.A_theta @ f)[m], 1 + 2 + 3, rtol=1e-12)
    assert np.allclose((P.B_theta @ f)[m], 1 - 2, rtol=1e-12)


@pytest.mark.parametrize("name", ["ex61_30_nu0.01_r3", "ex63_8"])
def test_example_operators_centred(name):
    """Examples 6.1/6.3: centred differences make the convection part
    skew-symmetric when the wind component is constant along its axis, and the
    right-hand side is scaled to ||C1 C2^T||_F = 1."""
    P = I.workload(name)
    nu = P.meta["nu"]
    L = I.laplacian(P.meta["N"], P.meta["dim"])
    if name.startswith("ex61"):
        # w_A = (1, 1): A - nu L is skew-symmetric
        K = P.A - nu * L
        assert abs(K + K.T).max() < 1e-9 * abs(K).max()
        # centred differences are exact on f = x away from the x-sides
        N = P.meta["N"]
        (x, y), h = _grid(N, 2)
        m = _interior([x, y], h)
        assert np.allclose((K @ (x - 2.0 * y))[m], 1.0 - 2.0, rtol=1e-12)
    nrm = np.linalg.norm(P.C1 @ P.C2.T)
    assert nrm == pytest.approx(1.0, rel=1e-12)


def test_rhs_factors_seeded_and_gaussian():
    a1, a2 = I.rhs_factors(4000, 3000, 4, 17)
    b1, b2 = I.rhs_factors(4000, 3000, 4, 17)
    c1, _ = I.rhs_factors(4000, 3000, 4, 18)
    assert np.array_equal(a1, b1) and np.array_equal(a2, b2)
    assert not np.array_equal(a1, c1)
    z = np.concatenate([a1.ravel(), a2.ravel()])
    assert abs(z.mean()) < 0.03 and abs(z.std() - 1.0) < 0.03


def test_diagonal_problem_closed_form_data():
    P = I.diagonal_problem(60, 5, 2, 3)
    assert len(np.unique(P.meta["a"])) == 5 and len(np.unique(P.meta["b"])) == 5
    assert np.array_equal(P.A.diagonal(), P.meta["a"])
    assert P.A.nnz == 60 and P.B.nnz == 60


def test_batched_sweep_distribution():
    """64 instances, N uniform in {64..384}, theta uniform in [1, 50],
    r in {1, 2, 4}; the same seed gives the same batch."""
    batch = I.batched_instances()
    assert len(batch) == 64
    Ns = [p.meta["N"] for p in batch]
    th = [p.theta for p in batch]
    rs = [p.r for p in batch]
    assert min(Ns) >= 64 and max(Ns) <= 384
    assert min(th) >= 1.0 and max(th) <= 50.0
    assert set(rs) <= {1, 2, 4} and len(set(rs)) == 3
    assert len(set(Ns)) > 40                                # uneven sizes
    for p in batch[:3]:
        assert p.n1 == p.meta["N"] ** 2 and p.A.nnz == 5 * p.n1 - 4 * p.meta["N"]
    again = I.batched_instances(count=3)
    for p, q in zip(batch[:3], again):
        assert p.meta["N"] == q.meta["N"] and p.theta == q.theta
        assert np.array_equal(p.C1, q.C1)


def test_operator_family_reassembles_the_convection_sweep():
    """The autograd path rebuilds A(theta) = A0 + theta A_theta and
    B(theta) on the host: at the problem's own theta it gives back A and B,
    and at another theta the generator's operators for that theta."""
    from paper_2311_16019_gb300.autograd import OperatorFamily
    P = I.workload("cd2d_32_r2")
    fam = OperatorFamily.from_problem(P)
    A, B = fam.at(P.theta)
    assert abs(A - P.A).max() < 1e-10 * abs(P.A).max()
    assert abs(B - P.B).max() < 1e-10 * abs(P.B).max()
    A3, _ = fam.at(3.0)
    want, _ = I.convdiff_2d(32, 3.0, lambda x, y: (x, y))
    assert abs(A3 - want).max() < 1e-10 * abs(want).max()
    assert A3.has_sorted_indices and B.has_sorted_indices
