"""The selection rule in the integer domain.

A draw is u = k * 2^-53 for the 53-bit integer k (the top 53 bits of two
Philox words).  The rule picks the first entry with u < C.  The CUDA path
compares k < ceil(C * 2^53) instead, computing the threshold once per table;
this holds exactly because the scaling by 2^53 is exact in binary floating
point.  These tests check the equivalence with exact rational arithmetic,
near thresholds and at the edges, and that the float computation of the
threshold (as the host writes it for pre-drawn tables) is the exact ceiling.
"""
import math
from fractions import Fraction

import numpy as np

TWO53 = 2 ** 53


def threshold(c: float) -> int:
    # the library's formula: ceil(c * 2^53) in double, then to an integer
    return math.ceil(c * 9007199254740992.0) if c > 0.0 else 0


def test_threshold_is_the_exact_ceiling():
    rng = np.random.default_rng(5)
    cs = np.concatenate([rng.random(20000), rng.random(2000) * 1e-6, [1.0, 0.5, 2.0 ** -53, 1.0 - 2.0 ** -53]])
    for c in cs.tolist():
        exact = math.ceil(Fraction(c) * TWO53)
        assert threshold(c) == exact


def test_integer_compare_equals_the_float_rule_near_thresholds():
    rng = np.random.default_rng(6)
    for c in rng.random(5000).tolist():
        t = threshold(c)
        for k in range(max(t - 3, 0), min(t + 3, TWO53)):
            u = k * 2.0 ** -53  # exact: k < 2^53
            assert Fraction(u) == Fraction(k, TWO53)
            assert (u < c) == (k < t)


def test_edges():
    # C = 1 selects every draw; C = 0 selects none; a cumulative table that
    # ends just below 1 leaves the top draws to the fallback (last nonzero)
    assert threshold(1.0) == TWO53
    assert all(k < threshold(1.0) for k in (0, TWO53 - 1))
    assert threshold(0.0) == 0
    c = 1.0 - 2.0 ** -53
    assert not (TWO53 - 1 < threshold(c))
    assert (TWO53 - 1) * 2.0 ** -53 >= c
