"""The library's true residual (spk_true_residual) and the mixed forms'
verification, through the C ABI.

spk_true_residual computes ||A X + X B - C1 C2^T||_F / ||C1 C2^T||_F for
X = X1 X2^T on the device in the factored form [A X1, X1, -C1][X2, B^T X2, C2]^T
with double-double Gram matrices.  It is compared with the oracle's
measurement (Householder QR of both factors, oracle/measure.py) and with a
closed form in which the three terms cancel to 1e-12 of their size."""
import numpy as np
import pytest
import scipy.sparse as sp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2311_16019_gb300 import inputs as I  # noqa: E402
from oracle import measure as M  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2311_16019_gb300 import build, spk
    build.build()
    return spk.load()


def spk():
    from paper_2311_16019_gb300 import spk as s
    return s


def host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("tol,d", [(1e-10, 0), (0.0, 12)])
def test_true_residual_against_oracle(tol, d):
    """A converged FP64 solve (relative residual ~1e-11) and an early one
    (~1e-2): the device value within 1e-4 (relative) of the oracle's."""
    P = I.workload("cd2d_64_r4")
    kw = dict(k=4, s=3200, maxit=400, p=20, tol=tol, seed=0)
    if d:
        kw.update(fixed_d=d, maxit=d)
    g = spk().solve(P.A, P.BT, P.C1, P.C2, **kw)
    num, den, rel = spk().true_residual(P.A, P.BT, P.C1, P.C2, g)
    want = M.true_residual(P.A, P.B, P.C1, P.C2, host(g.X1), host(g.X2))
    wden = M.lowrank_fro(P.C1, P.C2)
    print(f"d={g.iters}: device {rel:.6e} oracle {want:.6e}")
    assert abs(den - wden) <= 1e-13 * wden
    assert abs(rel - want) <= 1e-4 * want, (rel, want)
    assert abs(num - want * wden) <= 1e-4 * want * wden


def test_true_residual_closed_form_under_cancellation():
    """C1 = [A X1, X1, eps e1], C2 = [X2, B^T X2, e2] with integer operators
    and factors (every product exact in FP64): the residual of X = X1 X2^T is
    exactly -eps e1 e2^T, about 1e-12 of ||C1 C2^T||.  A Gram matrix in plain
    FP64 would resolve only ~1e-8 of the terms; the device value must match
    the closed form to 1e-6 relative."""
    P = I.workload("cd2d_64_r4")
    A, BT = P.A.tocsr().copy(), P.BT.tocsr().copy()
    A.data, BT.data = np.round(A.data), np.round(BT.data)     # integer stencils
    rng = np.random.default_rng(3)
    n = A.shape[0]
    ell = 3
    X1 = rng.integers(-50, 50, size=(n, ell)).astype(np.float64)
    X2 = rng.integers(-50, 50, size=(n, ell)).astype(np.float64)
    e1 = rng.integers(-3, 4, size=(n, 1)).astype(np.float64)
    e2 = rng.integers(-3, 4, size=(n, 1)).astype(np.float64)
    AX1, BX2 = A @ X1, BT @ X2
    C1n = np.hstack([AX1, X1])
    C2n = np.hstack([X2, BX2])
    big = M.lowrank_fro(C1n, C2n)
    eps = 1e-12 * big / (np.linalg.norm(e1) * np.linalg.norm(e2))
    C1 = np.hstack([C1n, eps * e1])
    C2 = np.hstack([C2n, e2])
    exact_num = eps * np.linalg.norm(e1) * np.linalg.norm(e2)
    den = M.lowrank_fro(C1, C2)
    sol = spk().SolveResult(0, 0, ell, True, 0.0, 0.0,
                            torch.as_tensor(X1, device="cuda"), torch.as_tensor(X2, device="cuda"),
                            [], [], 0, 0, 0, 0.0, 0.0, 0.0)
    num, gden, rel = spk().true_residual(A, BT, C1, C2, sol)
    print(f"closed form {exact_num / den:.6e}, device {rel:.6e}")
    assert abs(gden - den) <= 1e-12 * den
    assert abs(num - exact_num) <= 1e-6 * exact_num, (num, exact_num)


def test_mixed_fp32_reports_its_floor():
    """The FP32-basis form from the first iteration: the sketched estimate
    falls below tol 1e-9, the true residual stops near 1e-7 (the basis
    carries FP32 rounding the estimate cannot see; resuming the iteration
    does not lower it).  The solve must say so: status NOT_CONVERGED,
    converged False, and the measured true residual (equal to the oracle's
    measurement of the returned factors) above tol."""
    P = I.workload("cd2d_64_r4")
    g = spk().solve(P.A, P.BT, P.C1, P.C2, k=4, s=3200, maxit=400, p=20, tol=1e-9, seed=0,
                    precision="mixed_fp32")
    want = M.true_residual(P.A, P.B, P.C1, P.C2, host(g.X1), host(g.X2))
    print(f"mixed_fp32: d={g.iters} checks {g.hist_d} rel_rho={g.rel_rho:.2e} "
          f"true {g.true_rel_res:.3e} (oracle {want:.3e})")
    assert min(g.hist_rel) < 1e-9
    assert g.status == spk().SPK_ERR_NOT_CONVERGED and not g.converged
    assert g.true_rel_res > 1e-9
    assert abs(g.true_rel_res - want) <= 1e-4 * want


def test_mixed_fp32_with_fp64_start_reaches_tol():
    """The precision schedule: FP64 basis until the estimate is below 1e-4,
    FP32 after.  The early iterations' rounding is what the true residual
    keeps (measured with the oracle: switching at 1e-2 leaves ~1e-8, at 1e-4
    ~1e-9), so the form now reaches tol 1e-8 in the true residual (resuming
    once if the estimate's own gap needs it), and its X is within 1e-6 of
    the FP64 form's."""
    P = I.workload("cd2d_64_r4")
    kw = dict(k=4, s=3200, maxit=400, p=20, tol=1e-8, seed=0)
    f = spk().solve(P.A, P.BT, P.C1, P.C2, **kw)
    g = spk().solve(P.A, P.BT, P.C1, P.C2, precision="mixed_fp32", fp64_until=1e-4, **kw)
    want = M.true_residual(P.A, P.B, P.C1, P.C2, host(g.X1), host(g.X2))
    err = M.rel_error(host(g.X1), host(g.X2), host(f.X1), host(f.X2))
    print(f"switch at d={g.switch_d}, stop d={g.iters} (FP64 {f.iters}), checks {g.hist_d}, "
          f"true {g.true_rel_res:.3e} (oracle {want:.3e}), error vs FP64 {err:.2e}")
    assert 0 < g.switch_d < g.iters
    assert g.status == 0 and g.converged
    assert want < 1e-8 and abs(g.true_rel_res - want) <= 1e-4 * want
    assert err < 1e-6


def test_mixed_form_that_never_switches_is_the_fp64_solve():
    """fp64_until below any estimate: the mixed form never leaves FP64, and its
    factors are bit for bit those of the FP64 form (same kernels, same
    order; verification off so that both stop at the same check)."""
    P = I.workload("cd2d_24_r2")
    kw = dict(k=3, s=300, maxit=60, p=10, tol=1e-9, seed=2)
    f = spk().solve(P.A, P.BT, P.C1, P.C2, **kw)
    g = spk().solve(P.A, P.BT, P.C1, P.C2, precision="mixed_fp32", fp64_until=1e-300, verify=-1,
                    **kw)
    assert g.switch_d == -1 and f.true_rel_res == -1.0 and g.true_rel_res == -1.0
    assert g.iters == f.iters
    assert torch.equal(g.X1, f.X1) and torch.equal(g.X2, f.X2)


def test_verify_option_on_fp64_form():
    """verify=1 on the FP64 form: the true residual is reported and agrees
    with the oracle's measurement; verify=-1 skips it on a mixed form."""
    P = I.workload("lap32_r1")
    g = spk().solve(P.A, P.BT, P.C1, P.C2, k=2, s=600, maxit=300, p=10, tol=1e-8, seed=0,
                    verify=1)
    want = M.true_residual(P.A, P.B, P.C1, P.C2, host(g.X1), host(g.X2))
    assert g.converged == (want < 1e-8)
    assert abs(g.true_rel_res - want) <= 1e-4 * want
    print(f"lap32 verify=1: d={g.iters} checks {g.hist_d} true {g.true_rel_res:.3e}")
    h = spk().solve(P.A, P.BT, P.C1, P.C2, k=2, s=600, maxit=300, p=10, tol=1e-8, seed=0,
                    verify=-1, precision="mixed_fp32")
    assert h.true_rel_res == -1.0
