"""Pins of the oracle's sketch (Section 2.2) against definitions and known answers."""
import os

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import sketch as SK


def test_splitmix64_known_answers(golden_dir):
    rows = []
    for line in open(os.path.join(golden_dir, "splitmix64_kat.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append(tuple(int(t) for t in line.split()))
    for x0, idx, out in rows:
        got = int(SK.splitmix64_stream(x0, 1, start=idx)[0])
        assert got == out


def test_fwht_matches_hadamard_matrix():
    rng = np.random.default_rng(0)
    for q in range(0, 8):
        n = 2 ** q
        x = rng.standard_normal((n, 3))
        assert np.allclose(SK.fwht(x), sl.hadamard(n) @ x, rtol=0, atol=1e-12 * n)


def test_srht_dense_entries_definition():
    n, s = 37, 11
    S = SK.srht_dense(n, s, seed=5, sketch_id=1)
    rows, signs = SK.srht_draws(n, s, 5, 1)
    for j in range(s):
        for i in range(n):
            par = bin(int(rows[j]) & i).count("1") % 2
            assert S[j, i] == signs[i] * (-1) ** par / np.sqrt(s)


def test_srht_apply_exact_on_integers():
    rng = np.random.default_rng(1)
    n, s = 300, 40
    X = rng.integers(-1000, 1000, size=(n, 4)).astype(np.float64)
    S = SK.srht_dense(n, s, seed=9, sketch_id=0, scale=1.0)
    got = SK.srht_apply(X, s, seed=9, sketch_id=0, scale=1.0)
    assert np.array_equal(got, S @ X)


def test_draws_properties():
    n, s = 1000, 200
    rows, signs = SK.srht_draws(n, s, seed=3, sketch_id=0)
    assert rows.shape == (s,) and np.all(np.diff(rows) > 0)
    assert rows.min() >= 0 and rows.max() < SK.padded_length(n)
    assert set(np.unique(signs)) <= {-1, 1}
    # independent streams for the two sketches and the two sub-draws
    rows2, signs2 = SK.srht_draws(n, s, seed=3, sketch_id=1)
    assert not np.array_equal(rows, rows2) and not np.array_equal(signs, signs2)
    # the selection is the s smallest keys
    keys = SK.splitmix64_stream(SK.stream_state(3, 0, 0), SK.padded_length(n))
    assert keys[rows].max() < np.sort(keys)[s]


def test_full_srht_is_orthogonal():
    n = 64
    S = SK.srht_dense(n, n, seed=2, sketch_id=0, scale=1.0 / np.sqrt(n))
    assert np.allclose(S @ S.T, np.eye(n), atol=1e-13)
    x = np.random.default_rng(0).standard_normal(n)
    assert np.isclose(np.linalg.norm(SK.srht_apply(x, n, 2, 0, 1.0 / np.sqrt(n))),
                      np.linalg.norm(x), rtol=1e-13)


def test_embedding_distortion_on_krylov_basis():
    """Eq. (2.2): ||S v||^2 within (1 +- eps)||v||^2 on a Krylov space, s = 2 dim."""
    from paper_2311_16019_gb300 import inputs as I
    A = I.laplacian(24, 2)
    n = A.shape[0]
    rng = np.random.default_rng(4)
    K = [rng.standard_normal(n)]
    for _ in range(29):
        K.append(A @ K[-1] / np.linalg.norm(A @ K[-1]))
    Q, _ = np.linalg.qr(np.array(K).T)
    s = 4 * Q.shape[1]
    SQ = SK.srht_apply(Q, s, seed=11, sketch_id=0)
    sv = np.linalg.svd(SQ, compute_uv=False)
    # squared singular values = extreme distortions over the subspace
    assert sv.max() ** 2 < 1.0 + 0.9 and sv.min() ** 2 > 1.0 - 0.9


def test_dct_sketch_matches_its_dense_definition():
    """dct_apply (SciPy's DCT) equals the explicit cosine formula S[j, i] =
    sqrt(n/s) a_k cos(pi k (2i+1) / (2n)) e_i, k = rho_j."""
    for n, s in ((60, 17), (97, 40), (128, 128)):
        X = np.random.default_rng(n).standard_normal((n, 3))
        got = SK.dct_apply(X, s, seed=4, sketch_id=1)
        want = SK.dct_dense(n, s, seed=4, sketch_id=1) @ X
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def test_full_dct_sketch_is_orthogonal():
    """With s = n every row is selected: S = N E, an orthogonal matrix."""
    S = SK.dct_dense(90, 90, seed=2, sketch_id=0)
    assert np.abs(S.T @ S - np.eye(90)).max() < 1e-12


def test_dct_draws_properties():
    rows, signs = SK.dct_draws(1000, 123, seed=7, sketch_id=3)
    assert len(rows) == 123 and np.all(np.diff(rows) > 0)
    assert rows.min() >= 0 and rows.max() < 1000
    assert set(np.unique(signs)) <= {-1, 1}
    # the same sign stream as the SRHT of the same length
    _, s2 = SK.srht_draws(1000, 5, seed=7, sketch_id=3)
    assert np.array_equal(signs, s2)
