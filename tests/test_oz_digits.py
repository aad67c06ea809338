"""Exactness conditions of the digit-slice products used by the tensor-core 2-RDM
Gram and the FORTE_OZ64 alpha-beta sigma, checked on the CPU in integer
arithmetic (no GPU): the balanced base-256 digits reconstruct the fixed-point
value, every digit is an integer that BF16 holds exactly, the level sums over
K <= 64 products stay inside the ranges where the FP32 accumulator and the
magic-number rounding of the epilogue are exact, and the dropped levels weigh
at most 2^-49.99 of K times the product of the two operand bounds."""
import itertools

import numpy as np

XBITS = 45
K = 64


def digits(X):
    """Six balanced digits of |X| <= 2^45: add 0x80 to the five low bytes, read them back."""
    Y = X + 0x8080808080
    d = [Y >> 40] + [((Y >> (8 * (5 - i))) & 0xFF) - 128 for i in range(1, 6)]
    return d


def test_digits_reconstruct_and_stay_in_range():
    rng = np.random.default_rng(0)
    xs = [0, 1, -1, 2 ** XBITS, -(2 ** XBITS), 2 ** XBITS - 1, -(2 ** XBITS) + 1, 0x7F7F7F7F7F, -0x8080808080]
    xs += [int(v) for v in rng.integers(-(2 ** XBITS), 2 ** XBITS + 1, size=20000)]
    for X in xs:
        d = digits(X)
        assert sum(di * 256 ** (5 - i) for i, di in enumerate(d)) == X
        assert -32 <= d[0] <= 33 and all(-128 <= di <= 127 for di in d[1:])
        # an integer of at most 8 significant bits is exact in BF16 (8-bit significand)
        for di in d:
            m = abs(di)
            while m and m % 2 == 0:
                m //= 2
            assert m < 256


def test_level_sums_fit_the_exact_ranges():
    # worst case magnitudes: |d_1| <= 33 (the bound 32 plus the carry of 2^45
    # itself), |d_i| <= 128 otherwise
    dmax = [33] + [128] * 5
    for t in range(2, 9):
        pairs = [(i, t - i) for i in range(1, 7) if 1 <= t - i <= 6]
        bound = K * sum(dmax[i - 1] * dmax[j - 1] for i, j in pairs)
        # FP32 accumulation is exact below 2^24; the epilogue's magic-number
        # rounding needs |L| < 2^22 (1.5 2^23) for t <= 6 and < 2^23 (1.5 2^24) for t = 7, 8
        assert bound < 2 ** 24
        assert bound < (2 ** 22 if t <= 6 else 2 ** 23), (t, bound)


def test_dropped_levels_weigh_about_2_to_minus_50():
    dmax = [33] + [128] * 5
    dropped = 0
    for i, j in itertools.product(range(1, 7), repeat=2):
        if i + j > 8:
            dropped += K * dmax[i - 1] * dmax[j - 1] * 256 ** (12 - i - j)
    assert dropped < 2.0 ** -49.99 * K * 2 ** (2 * XBITS)


def test_folded_sum_fits_64_bits():
    # units of 2^6 L_8 = 2^38 in the product X_a X_b: |sum_k X_a X_b| <= K 2^90
    assert K * 2 ** (2 * XBITS) // 2 ** 38 < 2 ** 63
