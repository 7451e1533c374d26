"""The arithmetic of the error-free splitting behind the tensor-core FP64
products (Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59 (2012)), as the
kernels carry it out on the integer pipe, re-done here in Python integers and
IEEE doubles: the balanced base-2^7 digits taken from an FP64 bit pattern,
their exactness in BF16, the int8 widening by an FP32 subtraction, the bound
on every tensor-memory accumulator, and the exact recombination of the
weight levels in two 64-bit integers.  A slip in any of these (a digit
range, a bias, a shift, a level weight) fails one of these tests."""
import math
import struct

import numpy as np
import pytest


def f64_bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def digits8(x: float, e: int):
    """Balanced base-2^7 digits of N = rint(x 2^(56-e)), |x| < 2^e, from the
    FP64 bit pattern: the same steps as the device routine."""
    u = f64_bits(x)
    E = (u >> 52) & 0x7FF
    N = 0
    if E != 0:
        M = (u & ((1 << 52) - 1)) | (1 << 52)
        sh = E - 1023 - e + 4
        assert sh <= 3
        if sh >= 0:
            N = M << sh
        elif sh > -54:
            N = (M + (1 << (-sh - 1))) >> (-sh)
        if u >> 63:
            N = -N
    n = [0] * 8
    for p in range(7, 0, -1):
        d = ((N + 64) & 127) - 64
        n[p] = d
        N = (N - d) >> 7
    n[0] = N
    return n


def exp_above(x: float) -> int:
    """e with 2^e > |x| from the bit pattern (0 for 0)."""
    a = f64_bits(x) & ~(1 << 63)
    return ((a >> 52) & 0x7FF) - 1022 if a else 0


def bf16_bits_of_int(n: int) -> int:
    if n == 0:
        return 0
    a = abs(n)
    pos = a.bit_length() - 1
    return (0x8000 if n < 0 else 0) | ((127 + pos) << 7) | ((a << (7 - pos)) & 0x7F)


def bf16_value(b: int) -> float:
    return struct.unpack("<f", struct.pack("<I", b << 16))[0]


def values(rng, k):
    out = []
    for _ in range(k):
        kind = rng.integers(4)
        if kind == 0:
            out.append(float(rng.uniform(-1, 1)))
        elif kind == 1:
            out.append(float(rng.uniform(-1, 1) * 10.0 ** rng.uniform(-30, 30)))
        elif kind == 2:
            out.append(float(rng.choice([1.0, -1.0]) * (1 - 2.0 ** -53)))
        else:
            out.append(0.0)
    return out


def test_digits_reconstruct_to_57_bits_with_their_ranges():
    rng = np.random.default_rng(1)
    for x in values(rng, 20000):
        e = exp_above(x)
        assert abs(x) < 2.0 ** e
        n = digits8(x, e)
        assert abs(n[0]) <= 128 and all(-64 <= d <= 63 for d in n[1:])
        rec = sum(math.ldexp(d, e - 7 * (p + 1)) for p, d in enumerate(n))
        assert abs(rec - x) <= math.ldexp(1.0, e - 57) * (1 + 1e-12)


def test_leading_digit_of_orthonormal_entries_fits_int8_with_bias():
    # entries of Q (|q| <= 1) split with e = 1: |n_1| <= 64, so n + 128 fits a byte
    rng = np.random.default_rng(2)
    for q in list(rng.uniform(-1, 1, 5000)) + [1.0, -1.0, 1 - 2.0 ** -53]:
        n = digits8(float(q), 1)
        assert abs(n[0]) <= 64
        assert all(0 <= d + 128 <= 255 for d in n)


@pytest.mark.parametrize("n", list(range(-255, 256)))
def test_bf16_pattern_of_small_integers_is_exact(n):
    assert bf16_value(bf16_bits_of_int(n)) == n


def test_int8_widening_by_an_fp32_subtraction():
    # 2^23 + u is exact in FP32; minus 2^23 + 128 gives u - 128; the upper
    # half of that FP32 is the BF16 pattern of the digit
    for u in range(256):
        f = struct.unpack("<f", struct.pack("<I", 0x4B000000 | u))[0]
        v = np.float32(f) - np.float32(8388736.0)
        assert float(v) == u - 128
        upper = struct.unpack("<I", struct.pack("<f", float(v)))[0] >> 16
        assert bf16_value(upper) == u - 128


def test_accumulators_stay_exact_in_fp32():
    # general product: a level L (0-based) sums pairs (p, q), p + q = L, over
    # a K range of 256; whitening: each accumulator holds one pair over 256
    lead, rest = 128, 64
    worst_level = max(
        sum((lead if p == 0 else rest) * (lead if q == 0 else rest)
            for p in range(8) for q in range(8) if p + q == L)
        for L in range(8))
    assert 256 * worst_level < 2 ** 24
    assert 256 * 64 * 128 <= 2 ** 21          # one Q slice (|n| <= 64) x one B digit
    # FP32 sums of integers below 2^24 are exact whatever the order
    rng = np.random.default_rng(3)
    terms = rng.integers(-worst_level, worst_level + 1, size=256).astype(np.float32)
    assert float(np.sum(terms, dtype=np.float32)) == float(np.sum(terms.astype(np.int64)))


def test_levels_recombine_exactly_in_two_64_bit_integers():
    # hi = sum_{L<4} lev_L 2^(7 (3-L)), lo = sum_{L>=4} lev_L 2^(7 (7-L));
    # value = hi 2^-35 + lo 2^-63 equals sum_L lev_L 2^(-7 (L+2)) exactly
    rng = np.random.default_rng(4)
    for _ in range(2000):
        lev = [int(v) for v in rng.integers(-(2 ** 24), 2 ** 24, size=8)]
        hi = sum(lev[L] << (7 * (3 - L)) for L in range(4))
        lo = sum(lev[L] << (7 * (7 - L)) for L in range(4, 8))
        assert abs(hi) < 2 ** 53 and abs(lo) < 2 ** 53     # exact in FP64
        from fractions import Fraction
        exact = sum(Fraction(lev[L], 2 ** (7 * (L + 2))) for L in range(8))
        assert Fraction(hi, 2 ** 35) + Fraction(lo, 2 ** 63) == exact


def test_splitting_a_dot_product_matches_the_exact_sum():
    # one dot product through the whole scheme (digits, the 36 kept pairs,
    # level sums, recombination) against the exact rational dot product
    from fractions import Fraction
    rng = np.random.default_rng(5)
    K = 200
    a = rng.standard_normal(K) * 3.0
    b = rng.standard_normal(K) * 0.01
    ea = exp_above(float(np.max(np.abs(a))))
    eb = exp_above(float(np.max(np.abs(b))))
    da = [digits8(float(x), ea) for x in a]
    db = [digits8(float(x), eb) for x in b]
    lev = [0] * 8
    for p in range(8):
        for q in range(8 - p):
            lev[p + q] += sum(da[k][p] * db[k][q] for k in range(K))
    hi = sum(lev[L] << (7 * (3 - L)) for L in range(4))
    lo = sum(lev[L] << (7 * (7 - L)) for L in range(4, 8))
    got = math.ldexp(float(hi), ea + eb - 35) + math.ldexp(float(lo), ea + eb - 63)
    exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
    scale = 2.0 ** (ea + eb)
    assert abs(Fraction(got) - exact) <= Fraction(K * 2.0 ** -55 * scale) + Fraction(abs(got) * 2.0 ** -52)
