"""Pins of the s-PKSM oracle (Algorithm 1) to closed forms, textbook routines,
the paper's identities and the values the paper prints."""
import os

import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp

from paper_2311_16019_gb300 import inputs as I
from oracle import spkms as SP, arnoldi as AR, tpkms as TP, measure as M, adjoint as ADJ
from oracle.linalg import qr_pos, right_solve_upper, left_solve_upper, block_hessenberg
from oracle.sketch import Sketch


def _run(P, **kw):
    opts = dict(k=2, s=4 * 40, tol=0.0, maxit=20, p=1, seed=0)
    opts.update(kw)
    return SP.spkms(P.A, P.BT, P.C1, P.C2, **opts)


def test_qr_pos_convention():
    A = np.random.default_rng(0).standard_normal((30, 4))
    Q, R = qr_pos(A)
    assert np.all(np.diag(R) > 0) and np.allclose(Q @ R, A) and np.allclose(Q.T @ Q, np.eye(4))


@pytest.mark.parametrize("r", [1, 2])
def test_P1_diagonal_closed_form(r):
    """A, B diagonal with m distinct values: the block Krylov spaces are full
    after m steps and X_ij = (C1 C2^T)_ij / (a_i + b_j) exactly."""
    m = 6
    P = I.diagonal_problem(48, m, r, seed=3)
    res = _run(P, k=2, s=48 * 0 + 64, maxit=m, trunc_tol=1e-14)
    a, b = P.meta["a"], P.meta["b"]
    X = (P.C1 @ P.C2.T) / (a[:, None] + b[None, :])
    err = np.linalg.norm(res["X1"] @ res["X2"].T - X) / np.linalg.norm(X)
    assert err < 1e-10, err
    assert res["rel_rho"] < 1e-10


def test_P2_dense_bartels_stewart():
    P = I.workload("cd2d_24_r2")
    res = SP.spkms(P.A, P.BT, P.C1, P.C2, k=3, s=600, tol=1e-10, maxit=150, p=1, seed=1)
    assert res["converged"]
    X = ADJ.dense_solve(P.A, P.B, P.C1, P.C2)
    err = np.linalg.norm(res["X1"] @ res["X2"].T - X) / np.linalg.norm(X)
    # residual 1e-10 relative; A's condition number ~ 1e2 -> error ~ 1e-8 at most
    assert err < 1e-7, err
    assert M.true_residual(P.A, P.B, P.C1, P.C2, res["X1"], res["X2"]) < 5e-10


@pytest.mark.parametrize("kind", ["identity", "full_srht", "full_dct"])
@pytest.mark.parametrize("k", [1, 3])
def test_P3_reduction_to_galerkin(kind, k):
    """With an orthogonal sketch (S = I, or the SRHT with s = n' = n) the
    sketched-and-truncated approximation equals full Arnoldi's Galerkin one
    for any k (Section 2.3 RGS equivalence; Eq. (3.7)) and rho = ||R||_F."""
    P = I.workload("cd2d_16_r2")  # n = 256 = n'
    d = 12
    if kind == "identity":
        res = _run(P, k=k, s=256, maxit=d, sketch="identity", store_basis=True, trunc_tol=0)
    elif kind == "full_dct":
        res = _run(P, k=k, s=256, maxit=d, sketch="dct", store_basis=True, trunc_tol=0)
    else:
        res = _run(P, k=k, s=256, maxit=d, store_basis=True, trunc_tol=0)
    g = AR.galerkin(P.A, P.BT, P.C1, P.C2, d)
    X = SP.dense_solution(res)
    Xg = g["X1"] @ g["X2"].T
    assert np.linalg.norm(X - Xg) / np.linalg.norm(Xg) < 1e-10
    R = P.A @ X + X @ P.B - P.C1 @ P.C2.T
    assert abs(res["rho"] - np.linalg.norm(R)) < 1e-10 * np.linalg.norm(P.C1 @ P.C2.T)
    assert abs(res["rho"] - g["rho"]) < 1e-9 * g["rho"] + 1e-14


def test_P4_rho_equals_sketched_residual_bruteforce():
    """Eq. (3.5): ||S_U R S_V^T||_F = rho, with the whitened subdiagonal
    hhat = tau_{d+1} h_{d+1,d} tau_d^{-1}; the printed h_{d+1,d} does not."""
    P = I.workload("cd2d_24_r2")
    d = 10
    res = _run(P, k=2, s=150, maxit=d, store_basis=True)
    X = SP.dense_solution(res)
    R = P.A @ X + X @ P.B - P.C1 @ P.C2.T
    SU = res["SU"].dense()
    SV = res["SV"].dense()
    brute = np.linalg.norm(SU @ R @ SV.T)
    assert abs(brute - res["rho"]) < 1e-9 * brute
    # the printed (unwhitened) subdiagonal gives a different number
    m = d * 2
    Y = res["Y"]
    alt = np.sqrt(np.linalg.norm(res["H"][(d + 1, d)] @ Y[m - 2:, :]) ** 2
                  + np.linalg.norm(Y[:, m - 2:] @ res["G"][(d + 1, d)].T) ** 2)
    assert abs(alt - brute) > 1e-3 * brute


def test_P5_polynomial_exactness():
    """Eq. (4.11): Uhat_d p(H~_d) E_1 beta_1 = p(A) C1 for deg p <= d-1."""
    P = I.workload("cd2d_24_r2")
    d = 8
    res = _run(P, k=2, s=120, maxit=d, store_basis=True)
    r = 2
    m = d * r
    Ud = np.hstack([res["U_blocks"][j] for j in range(1, d + 1)])
    Uhat = right_solve_upper(Ud, res["T_U"][:m, :m])
    Ht = res["Ht"]
    v = np.zeros((m, r))
    v[:r] = res["beta1"]
    w = P.C1.copy()
    for j in range(d):
        lhs = Uhat @ v
        assert np.linalg.norm(lhs - w) < 1e-9 * np.linalg.norm(w), j
        v = Ht @ v
        w = P.A @ w


def test_P6_sketched_arnoldi_relation_and_bordering():
    """Proposition 2.1 (Eqs. (2.5)-(2.6)) with the stored basis; T is the R factor of
    S U_{d+1}; Section 5 bordering update equals T H T^{-1} (with the
    tau_{d+1}^{-1} reading of its last term)."""
    P = I.workload("cd2d_24_r2")
    d, r = 9, 2
    res = _run(P, k=3, s=120, maxit=d, store_basis=True, bordering=True)
    m = d * r
    U = np.hstack([res["U_blocks"][j] for j in range(1, d + 2)])
    SU = res["SU"].dense()
    Qf, Tf = qr_pos(SU @ U)
    assert np.allclose(Tf, res["T_U"], rtol=0, atol=1e-10 * np.abs(Tf).max())
    T = res["T_U"]
    Hd = block_hessenberg(res["H"], d, r)[:m, :m]
    TH = T[:m, m:]
    hn = res["H"][(d + 1, d)]
    RH = left_solve_upper(T[:m, :m], TH @ hn)
    Ed = np.zeros((m, r)); Ed[m - r:] = np.eye(r)
    lhs = SU @ P.A @ U[:, :m]
    rhs = SU @ U[:, :m] @ (Hd + RH @ Ed.T) + res["Q_U"][:, m:] @ T[m:, m:] @ hn @ Ed.T
    assert np.linalg.norm(lhs - rhs) < 1e-9 * np.linalg.norm(lhs)
    assert res["Q_U"][:, m:].T @ (SU @ U[:, :m]) == pytest.approx(np.zeros((r, m)), abs=1e-9)
    checks = res["bordering"]["checks"]
    assert len(checks) == 2 * (d - 1)
    for key, dd, diff, scale in checks:
        assert diff < 1e-9 * scale, (key, dd, diff, scale)


def test_P6b_printed_bordering_term_is_a_garble():
    """The last term of Hhat_new printed with tau_d^{-1} disagrees with
    T H T^{-1} whenever tau_d != tau_{d+1}."""
    P = I.workload("cd2d_24_r2")
    d, r = 5, 2
    res = _run(P, k=3, s=120, maxit=d + 1, store_basis=True)
    T = res["T_U"]
    m = d * r
    st = SP.SideState(P.A, 3, res["SU"], r, {}, res["H"], res["Q_U"], T[:m + r, :m + r],
                      None, None, False)
    Ht_d, _ = SP.projected_matrix(st, d)
    H_col = block_hessenberg(res["H"], d + 1, r)[:m, m:m + r]
    good = SP.bordering_update(Ht_d, T[:m + r, :m + r], H_col, res["H"][(d + 1, d)],
                               res["H"][(d + 1, d + 1)], r)
    direct = right_solve_upper(T[:m + r, :m + r] @ block_hessenberg(res["H"], d + 1, r)[:m + r, :m + r],
                               T[:m + r, :m + r])
    assert np.allclose(good, direct, atol=1e-9 * np.abs(direct).max())
    TH = T[:m, m:m + r]
    tau_d = T[m - r:m, m - r:m]
    printed = good[:m, m:].copy()
    printed += (right_solve_upper(TH @ res["H"][(d + 1, d + 1)], tau_d)
                - right_solve_upper(TH @ res["H"][(d + 1, d + 1)], T[m:m + r, m:m + r]))
    assert not np.allclose(printed, direct[:m, m:], atol=1e-6 * np.abs(direct).max())


def test_c5_initial_T_reading():
    """C1 = Uhat_d E_1 beta_1 (Eq. (3.4)) holds with T_{U,1} = R(S_U U_1) and
    beta_1 = T_{U,1} ell; it fails with the printed T_{U,1} = beta_1."""
    P = I.workload("cd2d_24_r2")
    res = _run(P, k=2, s=120, maxit=3, store_basis=True)
    U1 = res["U_blocks"][1]
    T1 = res["T_U"][:2, :2]
    assert np.allclose(right_solve_upper(U1, T1) @ res["beta1"], P.C1, atol=1e-10)
    assert not np.allclose(right_solve_upper(U1, res["beta1"]) @ res["beta1"], P.C1, atol=1e-3)


def test_c3_scale_invariance():
    """X does not depend on a scalar multiple c S of the sketch; rho scales by c^2."""
    P = I.workload("cd2d_24_r2")
    a = _run(P, k=2, s=120, maxit=10)
    b = _run(P, k=2, s=120, maxit=10, sketch_scale=np.sqrt(120 / 576.0) / np.sqrt(120))
    c2 = (np.sqrt(120 / 576.0) / np.sqrt(120) * np.sqrt(120)) ** 2
    assert M.rel_error(b["X1"], b["X2"], a["X1"], a["X2"]) < 1e-10
    assert b["rho"] == pytest.approx(c2 * a["rho"], rel=1e-9)
    assert b["rel_rho"] == pytest.approx(a["rel_rho"], rel=1e-9)


def test_P8_symmetry():
    P = I.workload("lap16_r1")
    res = SP.spkms(P.A, P.BT, P.C1, P.C1, k=2, s=128, tol=1e-9, maxit=80, p=1,
                   seed=0, same_sketch=True)
    X = res["X1"] @ res["X2"].T
    # identical recurrences on both sides: U = V, T_U = T_V, H = G exactly
    assert np.array_equal(res["T_U"], res["T_V"])
    assert all(np.array_equal(res["H"][key], res["G"][key]) for key in res["H"])
    assert np.abs(X - X.T).max() < 1e-12 * np.abs(X).max()


def test_P9_two_pass_replay_is_exact():
    P = I.workload("cd2d_24_r2")
    res = _run(P, k=3, s=120, maxit=12, store_basis=True)
    assert res["replay_maxdiff"] == 0.0
    # and the recovered factors reproduce the dense solution up to truncation
    X = SP.dense_solution(res)
    assert np.linalg.norm(res["X1"] @ res["X2"].T - X) < 1e-10 * np.linalg.norm(X)


def test_P10_tpkms_residual_bound():
    """Proposition 3.1: ||R_tr||_F <= sqrt(dr)(||Y E_d g^T|| + ||h E_d^T Y||)."""
    P = I.workload("cd2d_24_r2")
    for d in (5, 10, 15):
        res = TP.tpkms(P.A, P.BT, P.C1, P.C2, kA=2, kB=3, tol=0.0, maxit=d)
        X = res["X1"] @ res["X2"].T
        R = P.A @ X + X @ P.B - P.C1 @ P.C2.T
        assert np.linalg.norm(R) <= res["hist"][-1][1] * (1 + 1e-12)


def test_P11_example_4_2_arnoldi_relation():
    """Example 4.2's deterministic part: for the n = 30 Toeplitz matrix and
    b = ones/sqrt(n), the QR of the Krylov matrix gives A V(:,1:d-1) = V H with
    H = R(1:d,2:d) R(1:d-1,1:d-1)^{-1}; full Arnoldi must produce the same H
    (up to the column signs fixed by the positive-diagonal convention)."""
    n = 30
    col = np.zeros(n); col[:3] = [3, -1, -0.5]
    row = np.zeros(n); row[:3] = [3, 1, 1]
    A = -sl.toeplitz(col, row)
    b = np.ones(n) / np.sqrt(n)
    K = [b]
    for _ in range(4):
        K.append(A @ K[-1])
    K = np.array(K).T
    d = K.shape[1]
    V, R = qr_pos(K)
    H = R[:d, 1:d] @ np.linalg.inv(R[:d - 1, :d - 1])
    assert np.allclose(A @ V[:, :d - 1], V @ H, atol=1e-12)
    blocks, Hb, beta, r = AR.block_arnoldi(A, b, d - 1)
    Ha = block_hessenberg(Hb, d - 1, 1)
    Va = np.hstack([blocks[j] for j in range(1, d + 1)])
    assert np.allclose(Va, V, atol=1e-12)
    assert np.allclose(Ha, H, atol=1e-11)
    assert beta[0, 0] == pytest.approx(1.0)


def test_P12_memory_tables(golden_dir):
    for line in open(os.path.join(golden_dir, "memory_tables.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        t = line.split()
        if t[0] == "full":
            assert AR.memory_vectors_full(int(t[2]), int(t[1])) == int(t[3])
        elif t[0] == "spkms":
            assert AR.memory_vectors_spkms(int(t[1])) == int(t[2])
        else:
            assert AR.memory_vectors_tpkms(int(t[2]), int(t[3]), int(t[1])) == int(t[4])


def test_true_residual_measure_resolves_cancellation():
    """The oracle's true residual (Householder QR of both factors) against a
    closed form in which the terms cancel to 1e-10 of their size: integer
    operator and factors make A X1 and B^T X2 exact, and with
    C1 = [A X1, X1, eps e1], C2 = [X2, B^T X2, e2] the residual of
    X = X1 X2^T is exactly -eps e1 e2^T.  A Gram-trace expansion would
    return noise of order 1e-8 of the terms here."""
    P = I.workload("cd2d_32_r2")
    A, BT = P.A.tocsr().copy(), P.BT.tocsr().copy()
    A.data, BT.data = np.round(A.data), np.round(BT.data)     # integer stencils
    rng = np.random.default_rng(3)
    n = A.shape[0]
    X1 = rng.integers(-50, 50, size=(n, 3)).astype(np.float64)
    X2 = rng.integers(-50, 50, size=(n, 3)).astype(np.float64)
    e1 = rng.integers(-3, 4, size=(n, 1)).astype(np.float64)
    e2 = rng.integers(-3, 4, size=(n, 1)).astype(np.float64)
    C1n, C2n = np.hstack([A @ X1, X1]), np.hstack([X2, BT @ X2])
    big = np.linalg.norm(C1n @ C2n.T)
    eps = 1e-10 * big / (np.linalg.norm(e1) * np.linalg.norm(e2))
    C1, C2 = np.hstack([C1n, eps * e1]), np.hstack([C2n, e2])
    exact = eps * np.linalg.norm(e1) * np.linalg.norm(e2) / np.linalg.norm(C1 @ C2.T)
    got = M.true_residual(A, BT.T, C1, C2, X1, X2)
    assert got == pytest.approx(exact, rel=1e-4)


def test_measure_helpers_against_dense():
    rng = np.random.default_rng(0)
    X1, X2 = rng.standard_normal((50, 3)), rng.standard_normal((40, 3))
    Z1, Z2 = rng.standard_normal((50, 4)), rng.standard_normal((40, 4))
    D = X1 @ X2.T - Z1 @ Z2.T
    assert M.lowrank_diff_fro(X1, X2, Z1, Z2) == pytest.approx(np.linalg.norm(D), rel=1e-13)
    A = sp.random(50, 50, density=0.1, random_state=1) + sp.identity(50)
    B = sp.random(40, 40, density=0.1, random_state=2) + sp.identity(40)
    C1, C2 = rng.standard_normal((50, 2)), rng.standard_normal((40, 2))
    R = A @ (X1 @ X2.T) + (X1 @ X2.T) @ B - C1 @ C2.T
    assert M.true_residual(A, B, C1, C2, X1, X2) == pytest.approx(
        np.linalg.norm(R) / np.linalg.norm(C1 @ C2.T), rel=1e-12)
    # probes: zero for the same product in another gauge, 1/2 for Z = 2X,
    # and a flipped sign is seen
    G = np.array([[2.0, 1.0, 0.0], [0.0, 1.0, 0.0], [1.0, 0.0, 3.0]])
    assert M.probe_errors(X1, X2, X1 @ G, X2 @ np.linalg.inv(G).T) < 1e-13
    assert M.probe_errors(X1, X2, 2 * X1, X2) == pytest.approx(0.5, rel=1e-12)
    S1 = rng.standard_normal((50, 3))
    assert M.probe_errors(S1, S1, S1, -S1) > 1.0


def test_adjoint_dense_gradient_by_finite_differences():
    P = I.workload("cd2d_8_r2")
    rng = np.random.default_rng(5)
    u, v = rng.standard_normal(P.n1), rng.standard_normal(P.n2)
    g = ADJ.dense_gradient(P.A, P.B, P.A_theta, P.B_theta, P.C1, P.C2, u, v)
    h = 1e-6
    L = lambda A, B, C1, C2: float(u @ ADJ.dense_solve(A, B, C1, C2) @ v)
    Lp = L(P.A + h * P.A_theta, P.B + h * P.B_theta, P.C1, P.C2)
    Lm = L(P.A - h * P.A_theta, P.B - h * P.B_theta, P.C1, P.C2)
    assert (Lp - Lm) / (2 * h) == pytest.approx(g["dtheta"], rel=1e-6)
    E = np.zeros_like(P.C1); E[3, 1] = 1.0
    fd = (L(P.A, P.B, P.C1 + h * E, P.C2) - L(P.A, P.B, P.C1 - h * E, P.C2)) / (2 * h)
    assert fd == pytest.approx(g["dC1"][3, 1], rel=1e-6)
    fd = (L(P.A, P.B, P.C1, P.C2 + h * E[:P.n2]) - L(P.A, P.B, P.C1, P.C2 - h * E[:P.n2])) / (2 * h)
    assert fd == pytest.approx(g["dC2"][3, 1], rel=1e-6)


def test_converged_lap32_matches_full_arnoldi_iterations():
    """Table 2's qualitative claim (Example 6.1): s-PKSM needs about as many
    iterations as full Arnoldi (within 5 %) at the same tolerance."""
    P = I.workload("lap32_r1")
    res = SP.spkms(P.A, P.BT, P.C1, P.C2, k=2, s=600, tol=1e-8, maxit=300, p=1, seed=0)
    g = AR.galerkin(P.A, P.BT, P.C1, P.C2, 300, tol=1e-8)
    assert res["converged"] and abs(res["d"] - g["d"]) <= 0.05 * g["d"] + 1
    assert M.true_residual(P.A, P.B, P.C1, P.C2, res["X1"], res["X2"]) < 5e-8


def _cd2d_small(N, r, seed):
    A, _ = I.convdiff_2d(N, 10.0, lambda x, y: (x, y))
    B, _ = I.convdiff_2d(N, 10.0, lambda x, y: (y, -x))
    C1, C2 = I.rhs_factors(A.shape[0], B.shape[0], r, seed)
    return A, B, sp.csr_matrix(B.T), C1, C2


def test_P13_galerkin_exact_when_krylov_space_is_everything():
    """Full block Arnoldi (Eq. (2.1)) on a non-normal operator: once d r = n
    the bases are square and orthogonal, so the Galerkin solution is the
    exact solution of Eq. (1.1) and the residual (3.6) vanishes."""
    A, B, BT, C1, C2 = _cd2d_small(7, 7, 5)          # n = 49 = 7 blocks of 7
    X = ADJ.dense_solve(A, B, C1, C2)
    g = AR.galerkin(A, BT, C1, C2, 7)
    assert np.linalg.norm(g["X1"] @ g["X2"].T - X) < 1e-12 * np.linalg.norm(X)
    assert g["rel"] < 1e-12


@pytest.mark.parametrize("r", [2, 3])
def test_P13b_sketched_exact_when_krylov_space_is_everything(r):
    """Algorithm 1 with a subsampled (not orthogonal) SRHT, s = 60 of n' = 64
    rows for n = 36: S is injective on R^n, so once U_d and V_d span R^n
    (d r = 36) the sketched Petrov-Galerkin condition S_U R S_V^T = 0 forces
    R = 0.  (k = 3 keeps T's condition number near 1e9 (r = 2) and 1e7
    (r = 3) at d r = n; with k = 2 and r = 2 it reaches 1e16 and the
    recovered X is lost to rounding.)"""
    A, B, BT, C1, C2 = _cd2d_small(6, r, 5)
    X = ADJ.dense_solve(A, B, C1, C2)
    d = 36 // r
    res = SP.spkms(A, BT, C1, C2, k=3, s=60, tol=0.0, maxit=d, p=d, seed=3, trunc_tol=0)
    assert np.linalg.norm(res["X1"] @ res["X2"].T - X) < 1e-11 * np.linalg.norm(X)
    assert res["rel_rho"] < 1e-12


def test_P14_tpkms_with_full_window_is_full_arnoldi():
    """Algorithm 2 with k_A, k_B >= d orthogonalises against every block, so
    its bases, H, G and X are full Arnoldi's (Section 2.1), and its residual
    bound (3.3) brackets the exact residual norm (3.6):
    ||R|| <= rho_tr / sqrt(dr) <= sqrt(2) ||R||."""
    P = I.workload("cd2d_16_r2")
    d = 10
    t = TP.tpkms(P.A, P.BT, P.C1, P.C2, kA=d, kB=d, tol=0.0, maxit=d)
    g = AR.galerkin(P.A, P.BT, P.C1, P.C2, d)
    Xt, Xg = t["X1"] @ t["X2"].T, g["X1"] @ g["X2"].T
    assert np.linalg.norm(Xt - Xg) < 1e-12 * np.linalg.norm(Xg)
    R = P.A @ Xg + Xg @ P.B - P.C1 @ P.C2.T
    assert g["rho"] == pytest.approx(np.linalg.norm(R), rel=1e-9)
    scaled = t["hist"][-1][1] / np.sqrt(d * P.r)
    assert g["rho"] * (1 - 1e-12) <= scaled <= np.sqrt(2) * g["rho"] * (1 + 1e-12)


def test_P15_truncated_arnoldi_relation_and_local_orthogonality():
    """Algorithm 2's truncated block Arnoldi: A U_d = U_{d+1} H_(d+1 x d) with
    H banded (k - 1 blocks above the diagonal), and each new block
    orthonormal against the k blocks it was orthogonalised against, but not
    against older ones."""
    P = I.workload("cd2d_16_r2")
    d, k, r = 12, 2, 2
    blocks, H, beta = TP._truncated(P.A, P.C1, k, d)
    Ud = np.hstack([blocks[j] for j in range(1, d + 1)])
    Ud1 = np.hstack([blocks[j] for j in range(1, d + 2)])
    Hb = block_hessenberg(H, d, r)
    assert np.linalg.norm(P.A @ Ud - Ud1 @ Hb) < 1e-13 * np.linalg.norm(P.A @ Ud)
    for (i, j) in H:
        assert j - k + 1 <= i <= j + 1
    assert np.allclose(blocks[1] @ beta, P.C1, atol=1e-13 * np.abs(P.C1).max())
    far = 0.0
    for j in range(2, d + 2):
        assert np.allclose(blocks[j].T @ blocks[j], np.eye(r), atol=1e-13)
        for i in range(max(1, j - k), j):
            assert np.abs(blocks[i].T @ blocks[j]).max() < 1e-13
        if j - k - 1 >= 1:
            far = max(far, np.abs(blocks[j - k - 1].T @ blocks[j]).max())
    assert far > 1e-3          # the truncation is real: older blocks are not orthogonal


def test_truncation_rule_is_the_best_low_rank_approximation():
    """Reading c7 (Section 5's low-rank factors of Y): keep the singular
    triplets with sigma_i > eps sigma_1 and split sqrt(Sigma) between the
    factors.  Y1 Y2^T is then the best rank-l approximation (Eckart-Young:
    spectral error sigma_{l+1}), Y1^T Y1 = Y2^T Y2 = Sigma_l, and the count
    follows the threshold exactly, on a matrix with known singular values."""
    rng = np.random.default_rng(11)
    m = 40
    Pm, _ = np.linalg.qr(rng.standard_normal((m, m)))
    Qm, _ = np.linalg.qr(rng.standard_normal((m, m)))
    sig = 0.5 * 10.0 ** (-np.arange(m) / 4.0)          # sigma_1 / sigma_40 = 1e9.75
    Y = (Pm * sig[None, :]) @ Qm.T
    for eps, ell in ((10 ** (-2.5 / 4), 3), (10 ** (-20.5 / 4), 21), (0.0, m)):
        Y1, Y2, s = SP.truncate(Y, eps)
        assert Y1.shape == (m, ell) and Y2.shape == (m, ell)
        assert np.allclose(s, sig, rtol=1e-5)
        E = Y - Y1 @ Y2.T
        tail = sig[ell] if ell < m else 0.0
        assert np.linalg.norm(E, 2) <= tail * (1 + 1e-6) + 1e-15
        assert np.allclose(Y1.T @ Y1, np.diag(sig[:ell]), atol=1e-13)
        assert np.allclose(Y2.T @ Y2, np.diag(sig[:ell]), atol=1e-13)


@pytest.mark.parametrize("s,d", [(400, 10), (500, 20)])
def test_P16_sketched_residual_bound_of_appendix_B(s, d):
    """Eq. (3.6) via Theorem B.3: the residual lies in span(U_{d+1}) x
    span(V_{d+1}) (Arnoldi relations), so rho = ||S_U R S_V^T||_F and ||R||_F
    differ at most by the extreme singular values of the sketched orthonormal
    bases, and (1+et)^-1 rho^2 <= ||R||^2 <= (1-et)^-1 rho^2 with
    et = eps (2 + eps), eps the measured embedding distortion of the two
    (d+1) r dimensional Krylov spaces (squared-norm definition, Eq. (2.2))."""
    P = I.workload("cd2d_24_r2")
    res = _run(P, k=2, s=s, maxit=d, p=d, store_basis=True)
    X = SP.dense_solution(res)
    R = P.A @ X + X @ P.B - P.C1 @ P.C2.T
    eps, lo, hi = 0.0, 1.0, 1.0
    for blocks, S in ((res["U_blocks"], res["SU"]), (res["V_blocks"], res["SV"])):
        basis = sl.orth(np.hstack([blocks[j] for j in range(1, d + 2)]))
        assert basis.shape[1] == (d + 1) * P.r
        sv = np.linalg.svd(S.dense() @ basis, compute_uv=False)
        eps = max(eps, float(np.max(np.abs(sv ** 2 - 1.0))))
        lo, hi = lo * sv.min(), hi * sv.max()
    rho, nR = res["rho"], np.linalg.norm(R)
    assert lo * nR * (1 - 1e-10) <= rho <= hi * nR * (1 + 1e-10)
    et = eps * (2 + eps)
    assert et < 1.0
    assert rho ** 2 / (1 + et) <= nR ** 2 <= rho ** 2 / (1 - et)


class _Fp32Operator:
    """A applied in float32 to a float32-rounded block: what a basis stored
    in FP32 and an FP32 SpMM give the recurrence."""

    def __init__(self, A):
        self.A = sp.csr_matrix(A, dtype=np.float32)

    def __matmul__(self, X):
        return (self.A @ np.asarray(X, dtype=np.float32)).astype(np.float64)


def test_fp32_basis_floor_is_inherent_to_the_method():
    """The mixed form (FP32 basis and SpMM, FP64 sketch side) is not in the
    paper.  With A applied in FP32 the Arnoldi relation (2.4) holds only to
    FP32 accuracy: the sketched estimate rho (3.5) still converges (it
    measures the projected problem), but the true residual stops near
    u_32-scale.  The oracle with an FP32 operator shows this floor, so the
    GPU mixed form's residual floor is the method's in that precision."""
    P = I.workload("cd2d_32_r2")
    kw = dict(k=4, s=1000, tol=1e-10, maxit=250, p=10, seed=0)
    ref = SP.spkms(P.A, P.BT, P.C1, P.C2, **kw)
    mixed = SP.spkms(_Fp32Operator(P.A), _Fp32Operator(P.BT), P.C1, P.C2, **kw)
    assert ref["converged"] and mixed["converged"]
    t_ref = M.true_residual(P.A, P.B, P.C1, P.C2, ref["X1"], ref["X2"])
    t_mix = M.true_residual(P.A, P.B, P.C1, P.C2, mixed["X1"], mixed["X2"])
    assert t_ref < 1e-10
    assert mixed["rel_rho"] < 1e-10
    assert 1e-8 < t_mix < 1e-6


def test_projected_spectra_leave_the_right_half_plane_past_convergence():
    """Section 4.1's caveat, measured: the field of values of H~_d can cross
    the imaginary axis although A's lies in the right half plane.  On the 3-D
    upwind problem (16^3, r = 2, k = 3, s = 1600) every eigenvalue of H~_d
    and G~_d has positive real part at d = 60 (rho/||beta1 beta2^T|| 2e-13),
    while past convergence some do not (d = 200).  This is why the GPU's
    sign-function solve checks trace(sign) = m and an adaptive schedule that
    overshoots backs off to an earlier, solvable check."""
    P = I.workload("cd3d_16_r2")
    neg = {}
    for d in (60, 200):
        res = SP.spkms(P.A, P.BT, P.C1, P.C2, k=3, s=1600, tol=0.0, maxit=d, p=d, seed=0,
                       recover=False)
        eh = np.linalg.eigvals(res["Ht"])
        eg = np.linalg.eigvals(res["Gt"])
        neg[d] = int(np.sum(eh.real < 0) + np.sum(eg.real < 0))
        if d == 60:
            assert res["rel_rho"] < 1e-12
    A = P.A.toarray()
    assert np.linalg.eigvalsh((A + A.T) / 2).min() > 0      # W(A) in the right half plane
    assert neg[60] == 0 and neg[200] > 0


def test_leading_block_of_the_projected_matrix_is_the_earlier_one():
    """H~_d = T_d H_d T_d^{-1} + T_H h_{d+1,d} tau_d^{-1} E_d^T (Eqs. (2.9)-(2.10))
    has H~_{d'} as its leading d'r x d'r block for every d' < d: T_d and H_d
    are upper triangular / Hessenberg with T_{d'}, H_{d'} in their corners,
    and the correction of H~_{d'} is exactly the (d'+1, d') coupling term of
    T_d H_d T_d^{-1} restricted to those rows.  The GPU's backtracking after
    an unsolvable check relies on this: it re-solves on a leading block
    instead of rebuilding an earlier H~."""
    P = I.workload("cd2d_24_r2")
    r, d = P.r, 16
    full = _run(P, k=3, s=300, maxit=d, p=d)
    for dp in (5, 11):
        part = _run(P, k=3, s=300, maxit=dp, p=dp)
        m = dp * r
        for key in ("Ht", "Gt"):
            lead = full[key][:m, :m]
            assert np.abs(lead - part[key]).max() < 1e-12 * np.abs(part[key]).max(), (key, dp)


@pytest.mark.parametrize("sketch,k,k_right", [("dct", 2, 2), ("srht", 2, 4), ("dct", 3, 1)])
def test_P4b_rho_bruteforce_other_sketches_and_windows(sketch, k, k_right):
    """Eq. (3.5) against ||S_U R S_V^T||_F formed densely, with the DCT sketch
    of Section 6 (s < n, not orthogonal) and with different truncations for
    the two spaces (Algorithm 1 takes one k; the spaces are independent)."""
    P = I.workload("cd2d_24_r2")
    d = 10
    res = _run(P, k=k, k_right=k_right, s=150, maxit=d, p=d, sketch=sketch, store_basis=True)
    X = SP.dense_solution(res)
    R = P.A @ X + X @ P.B - P.C1 @ P.C2.T
    brute = np.linalg.norm(res["SU"].dense() @ R @ res["SV"].dense().T)
    assert abs(brute - res["rho"]) < 1e-9 * brute
    # and X is the recovered solution of the two-pass step
    assert np.linalg.norm(res["X1"] @ res["X2"].T - X) < 1e-10 * np.linalg.norm(X)
