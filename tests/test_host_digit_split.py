"""The precision form's exact digit split, modelled in Python integers on the
host: the facts its GPU tests rely on, checked here from the definition
(no GPU, no code shared with the CUDA path).

A value a with split exponent e (|a| 2^-e < 1/2) is rounded to the 48-bit
integer F = round(|a| 2^(49-e)) and written as seven balanced base-128 digits
F = sum_s d_s 128^(6-s), d_0 in [0, 64], d_1..d_6 in [-64, 63]; a product a b
keeps the digit pairs of levels s + t <= 6 (28 of 49).  The tests check the
reconstruction, the digit ranges, the per-term error bound the GPU Gram and
update tests assert (8 * 2^-48 * max|a| max|b|), and the level-sum bound that
makes 512-row FP32 block sums exact."""
from fractions import Fraction

import numpy as np

U = Fraction(1, 2 ** 48)


def _fixed(a, e):
    # F = round(|a| 2^(49-e)), exact rational arithmetic, ties away from zero
    x = abs(Fraction(a)) * Fraction(2) ** (49 - e)
    F = int(x)
    if x - F >= Fraction(1, 2):
        F += 1
    return F


def _digits(F):
    d = [0] * 7
    for s in range(6, 0, -1):
        x = F % 128
        F //= 128
        if x >= 64:
            x -= 128
            F += 1
        d[s] = x
    d[0] = F
    return d


def _split_exp(cmax):
    # |v| < 2^(e-1) for the column's largest |v|: e = ilogb(cmax) + 2
    return int(np.floor(np.log2(cmax))) + 2 if cmax > 0 else 1


def _trunc_product(a, ea, b, eb):
    da, db = _digits(_fixed(a, ea)), _digits(_fixed(b, eb))
    sgn = (1 if a >= 0 else -1) * (1 if b >= 0 else -1)
    acc = Fraction(0)
    for s in range(7):
        for t in range(7 - s):
            acc += Fraction(da[s] * db[t], 128 ** (s + t + 2))
    return sgn * acc * Fraction(2) ** (ea + eb)


def test_digits_reconstruct_and_stay_in_range():
    rng = np.random.default_rng(1)
    for _ in range(3000):
        a = float(rng.standard_normal() * 10.0 ** rng.integers(-30, 30))
        e = _split_exp(abs(a)) + int(rng.integers(0, 3))
        F = _fixed(a, e)
        assert 0 <= F < 2 ** 48
        d = _digits(F)
        assert sum(x * 128 ** (6 - s) for s, x in enumerate(d)) == F
        assert 0 <= d[0] <= 64 and all(-64 <= x <= 63 for x in d[1:])
        assert all(abs(x) <= 64 for x in d)  # every digit exact in BF16, |d_s d_t| <= 2^12


def test_truncated_product_within_the_stated_bound():
    # the bound the GPU tests assert per term: 8 * 2^-48 * max|A_j| max|A_k|
    rng = np.random.default_rng(2)
    worst = Fraction(0)
    for _ in range(1500):
        cmax_a, cmax_b = 10.0 ** rng.uniform(-8, 8, 2)
        a = float(cmax_a * rng.uniform(-1, 1))
        b = float(cmax_b * rng.uniform(-1, 1))
        ea, eb = _split_exp(cmax_a), _split_exp(cmax_b)
        err = abs(Fraction(a) * Fraction(b) - _trunc_product(a, ea, b, eb))
        ratio = err / (8 * U * Fraction(cmax_a) * Fraction(cmax_b))
        worst = max(worst, ratio)
    assert worst <= 1, float(worst)


def test_all_63_digits_reach_the_level_bound_and_stay_exact():
    # the GPU exactness test's construction: F with every digit 63 gives level
    # sums (w + 1) 63^2 per row; over 512 rows level 4 passes 2^23 and level 6
    # stays below 2^24, inside the FP32 integer range that makes the block
    # sums exact; its dropped levels cost 2.97 * 2^-48 of the product, inside
    # the stated 8 * 2^-48
    F = sum(63 * 128 ** (6 - s) for s in range(7))
    assert _digits(F) == [63] * 7
    level = [(w + 1) * 63 * 63 * 512 for w in range(7)]
    assert level[4] > 2 ** 23 and max(level) < 2 ** 24
    assert 512 * 7 * 2 ** 12 < 2 ** 24  # any digits: 7 pairs per level, |d_s d_t| <= 2^12
    a = float(Fraction(F, 2 ** 47))  # |a| in [1, 2): split exponent 2
    exact = Fraction(a) ** 2
    drop = exact - _trunc_product(a, 2, a, 2)
    assert 0 < drop / exact < 3 * U
    assert drop <= 8 * U * exact
