"""Host-side setup of the differentiable solve, checked on the CPU: the
operators A(theta), B(theta)^T, A(theta)^T and B(theta) are held on the
union sparsity pattern of their two parts, and their values at any theta
are v0 + theta v_theta on that pattern (formed on the device by the
library's FP64 product).  Here: that pattern and those values reproduce the
host assembly X0 + theta X_theta entry for entry, for parts whose patterns
differ, overlap and cancel."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2311_16019_gb300 import inputs as I
from paper_2311_16019_gb300.autograd import OperatorFamily, union_pattern


def _assemble(shape, indptr, indices, v0, vt, theta):
    return sp.csr_matrix((v0 + theta * vt, indices, indptr), shape=shape)


@pytest.mark.parametrize("theta", [0.0, 0.37, -2.5, 10.0])
def test_union_pattern_reproduces_the_family(theta):
    P = I.workload("cd2d_16_r2")
    fam = OperatorFamily.from_problem(P)
    A, B = fam.at(theta)
    for X0, Xt, ref in [(fam.A0, fam.A_theta, A), (fam.B0.T, fam.B_theta.T, B.T),
                        (fam.A0.T, fam.A_theta.T, A.T), (fam.B0, fam.B_theta, B)]:
        shape, indptr, indices, v0, vt = union_pattern(X0, Xt)
        assert indptr.dtype == np.int32 and indices.dtype == np.int32
        M = _assemble(shape, indptr, indices, v0, vt, theta)
        assert abs(M - ref).max() == 0.0
        # sorted column indices within each row
        for i in range(shape[0]):
            row = indices[indptr[i]:indptr[i + 1]]
            assert np.all(np.diff(row) > 0)


def test_union_pattern_of_disjoint_and_cancelling_parts():
    rng = np.random.default_rng(4)
    X0 = sp.random(40, 40, density=0.1, random_state=rng, format="csr")
    Xt = sp.random(40, 40, density=0.1, random_state=rng, format="csr")
    Xt = Xt - X0     # overlapping entries, and entries where X0 + Xt cancels
    shape, indptr, indices, v0, vt = union_pattern(X0, Xt)
    pattern = (abs(X0) + abs(Xt)) != 0
    assert indptr[-1] == pattern.nnz
    for theta in (1.0, 0.5, -3.0):
        M = _assemble(shape, indptr, indices, v0, vt, theta)
        assert abs(M - (X0 + theta * Xt)).max() <= 1e-15
