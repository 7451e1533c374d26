"""Subsampled randomized trigonometric sketches (Section 2.2), oracle side.

The paper builds S = sqrt(s/n) D N E: E a random +-1 diagonal, N a
trigonometric transform (DFT, DCT or Walsh-Hadamard are all allowed), D a
random selection of s rows.  This restatement takes N = the Walsh-Hadamard
transform on n' = 2^ceil(log2 n) points (x zero-padded from n to n') and the
norm-preserving scale, so that

    S[j, i] = e_i * (-1)^popcount(rho_j & i) / sqrt(s),   i < n,

where rho_0 < rho_1 < ... < rho_{s-1} are the selected rows.  (The paper's
printed factor sqrt(s/n) would shrink norms by s/n; the solution X does not
depend on any scalar multiple of S -- T, beta and Y scale together -- and the
stopping test is taken relative to ||beta_1 beta_2^T||, so only the sketched
residual's units depend on the reading.)

The DCT sketch of the paper's experiments (Section 6) is also provided
(`dct_*`): N = the orthonormal DCT-II on the n rows themselves (no padding),
scale sqrt(n/s), rows drawn over [0, n) from the same streams.

Random draws (the paper leaves them unspecified) come from the SplitMix64
generator of Steele, Lea and Flood (OOPSLA 2014) as published by Vigna: the
i-th output of a generator whose state starts at x0 is
    z = x0 + (i+1) * 0x9E3779B97F4A7C15 (mod 2^64)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    out = z ^ (z >> 31).
Stream x0 = seed + (1 + 2*sketch_id + sub) * 0x632BE59BD9B4E019 (mod 2^64),
sub = 0 for row keys, 1 for signs.  Signs: e_i = 1 - 2*(out_i >> 63).  Rows:
the s indices in [0, n') with the smallest keys out_i (keys are distinct:
i -> out_i is injective), stored in ascending index order.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM = 0x632BE59BD9B4E019


def splitmix64_stream(x0: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start..start+count-1 of SplitMix64 started at state x0."""
    i = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(x0 % (1 << 64)) + (i + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_state(seed: int, sketch_id: int, sub: int) -> int:
    """Start state of the SplitMix64 stream of one sketch (sketch_id 0 for
    S_U, 1 for S_V) and one kind of draw (sub 0: row keys of D, 1: signs of
    E).  Section 2.2 leaves the random draws of D and E unspecified."""
    return (seed + (1 + 2 * sketch_id + sub) * _STREAM) % (1 << 64)


def padded_length(n: int) -> int:
    """n' = smallest power of two >= n."""
    p = 1
    while p < n:
        p *= 2
    return p


def srht_draws(n: int, s: int, seed: int, sketch_id: int):
    """(rows int64[s] ascending, signs int8[n]) of the SRHT for length n."""
    npad = padded_length(n)
    if not (1 <= s <= npad):
        raise ValueError("need 1 <= s <= n'")
    keys = splitmix64_stream(stream_state(seed, sketch_id, 0), npad)
    order = np.argsort(keys, kind="stable")
    rows = np.sort(order[:s]).astype(np.int64)
    sbits = splitmix64_stream(stream_state(seed, sketch_id, 1), n) >> np.uint64(63)
    signs = (1 - 2 * sbits.astype(np.int64)).astype(np.int8)
    return rows, signs


def _popcount_parity(a: np.ndarray) -> np.ndarray:
    """Parity of the number of set bits of each entry, one bit at a time:
    the Walsh-Hadamard entry H[j, i] (Sylvester ordering) is
    (-1)^parity(j & i), the N of Section 2.2's S = D N E."""
    a = a.astype(np.uint64)
    par = np.zeros(a.shape, dtype=np.uint64)
    while np.any(a):
        par ^= a & np.uint64(1)
        a = a >> np.uint64(1)
    return par


def srht_dense(n: int, s: int, seed: int, sketch_id: int, scale: float | None = None) -> np.ndarray:
    """The explicit s x n matrix S[j,i] = e_i (-1)^popcount(rho_j & i) * scale."""
    rows, signs = srht_draws(n, s, seed, sketch_id)
    if scale is None:
        scale = 1.0 / np.sqrt(s)
    i = np.arange(n, dtype=np.uint64)
    par = _popcount_parity(rows.astype(np.uint64)[:, None] & i[None, :])
    return (1.0 - 2.0 * par.astype(np.float64)) * signs[None, :].astype(np.float64) * scale


def fwht(x: np.ndarray) -> np.ndarray:
    """Unnormalised Walsh-Hadamard transform along axis 0 (length 2^q).

    y[c] = sum_i (-1)^popcount(c & i) x[i], by the standard butterfly.
    """
    y = np.array(x, dtype=np.float64, copy=True)
    n = y.shape[0]
    h = 1
    while h < n:
        y = y.reshape((n // (2 * h), 2, h) + y.shape[1:])
        a = y[:, 0].copy()
        b = y[:, 1].copy()
        y[:, 0] = a + b
        y[:, 1] = a - b
        y = y.reshape((n,) + y.shape[3:])
        h *= 2
    return y


def srht_apply(X: np.ndarray, s: int, seed: int, sketch_id: int, scale: float | None = None) -> np.ndarray:
    """S @ X for X of shape (n,) or (n, r): sign, pad, transform, select, scale."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    rows, signs = srht_draws(n, s, seed, sketch_id)
    npad = padded_length(n)
    Z = np.zeros((npad,) + X.shape[1:])
    Z[:n] = X * (signs.reshape((n,) + (1,) * (X.ndim - 1)))
    if scale is None:
        scale = 1.0 / np.sqrt(s)
    return fwht(Z)[rows] * scale


def dct_draws(n: int, s: int, seed: int, sketch_id: int):
    """(rows int64[s] ascending, signs int8[n]) of the DCT sketch: the same
    SplitMix64 streams as the SRHT, with the row keys taken over the n rows
    themselves (no padding)."""
    if not (1 <= s <= n):
        raise ValueError("need 1 <= s <= n")
    keys = splitmix64_stream(stream_state(seed, sketch_id, 0), n)
    order = np.argsort(keys, kind="stable")
    rows = np.sort(order[:s]).astype(np.int64)
    sbits = splitmix64_stream(stream_state(seed, sketch_id, 1), n) >> np.uint64(63)
    signs = (1 - 2 * sbits.astype(np.int64)).astype(np.int8)
    return rows, signs


def dct_dense(n: int, s: int, seed: int, sketch_id: int, scale: float | None = None) -> np.ndarray:
    """The explicit s x n DCT sketch (the paper's choice of N in its
    experiments, Section 6): S = scale * D N E with N the orthonormal DCT-II,
    N[k, i] = a_k cos(pi k (2 i + 1) / (2 n)), a_0 = sqrt(1/n), a_k = sqrt(2/n);
    scale sqrt(n/s) keeps norms in expectation (the reading of the printed
    constant, as for the SRHT)."""
    rows, signs = dct_draws(n, s, seed, sketch_id)
    if scale is None:
        scale = np.sqrt(n / s)
    k = rows.astype(np.float64)[:, None]
    i = np.arange(n, dtype=np.float64)[None, :]
    a = np.where(rows == 0, np.sqrt(1.0 / n), np.sqrt(2.0 / n))[:, None]
    return scale * a * np.cos(np.pi * k * (2.0 * i + 1.0) / (2.0 * n)) * signs[None, :]


def dct_apply(X: np.ndarray, s: int, seed: int, sketch_id: int, scale: float | None = None) -> np.ndarray:
    """S @ X for the DCT sketch: sign, orthonormal DCT-II (SciPy), select, scale."""
    import scipy.fft as sfft
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    rows, signs = dct_draws(n, s, seed, sketch_id)
    if scale is None:
        scale = np.sqrt(n / s)
    Z = X * (signs.reshape((n,) + (1,) * (X.ndim - 1)))
    return sfft.dct(Z, type=2, norm="ortho", axis=0)[rows] * scale


class Sketch:
    """S as an operator: kind 'srht', 'dct' or 'identity' (S = I_n, s = n)."""

    def __init__(self, n: int, s: int, seed: int, sketch_id: int, kind: str = "srht",
                 scale: float | None = None):
        self.n, self.kind = n, kind
        if kind == "identity":
            self.s = n
            self.scale = 1.0 if scale is None else scale
        elif kind == "srht":
            self.s = s
            self.seed, self.sketch_id = seed, sketch_id
            self.scale = (1.0 / np.sqrt(s)) if scale is None else scale
        elif kind == "dct":
            self.s = s
            self.seed, self.sketch_id = seed, sketch_id
            self.scale = np.sqrt(n / s) if scale is None else scale
        else:
            raise ValueError(kind)

    def __call__(self, X: np.ndarray) -> np.ndarray:
        """S X for the columns of X (Section 2.2)."""
        if self.kind == "identity":
            return np.array(X, dtype=np.float64) * self.scale
        if self.kind == "dct":
            return dct_apply(X, self.s, self.seed, self.sketch_id, self.scale)
        return srht_apply(X, self.s, self.seed, self.sketch_id, self.scale)

    def dense(self) -> np.ndarray:
        """The explicit s x n matrix S, for brute-force checks."""
        if self.kind == "identity":
            return np.eye(self.n) * self.scale
        if self.kind == "dct":
            return dct_dense(self.n, self.s, self.seed, self.sketch_id, self.scale)
        return srht_dense(self.n, self.s, self.seed, self.sketch_id, self.scale)
