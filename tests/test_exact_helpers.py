"""The exact fixed-point references the GPU delta and mass tests compare with:
pinned against rational arithmetic on the CPU, so a mistake in the helpers
cannot hide a mistake in the kernels."""
from fractions import Fraction

import numpy as np

from gpu_helpers import exact_l1_change, exact_sum

UNIT = Fraction(1, 2 ** 60)


def _trunc60(v):
    """floor(v * 2^60) * 2^-60 for a non-negative float, in rationals."""
    return Fraction(int(Fraction(float(v)) / UNIT)) * UNIT


def test_exact_helpers_equal_rational_sums():
    rng = np.random.default_rng(0xF1)
    for n in (1, 7, 1000):
        a = (rng.random(n) * rng.choice([1.0, 1e-3, 1e-8, 2.0 ** -40], n)).astype(np.float32)
        b = (rng.random(n) * rng.choice([1.0, 1e-3, 1e-8, 2.0 ** -40], n)).astype(np.float32)
        want = sum(abs(_trunc60(p) - _trunc60(q)) for p, q in zip(a, b))
        assert exact_l1_change(a, b) == float(want)  # one rounding, to nearest
        assert exact_sum(a) == float(sum(_trunc60(p) for p in a))


def test_scores_at_or_above_2_pow_minus_37_are_exact():
    """Every float >= 2^-37 is a multiple of 2^-60, so nothing is truncated."""
    v = np.array([2.0 ** -37, 0.15 / 2 ** 31, 1.0 / 3.0, 0.999999], np.float32)
    for x in v:
        assert _trunc60(x) == Fraction(float(x))
    assert exact_sum(v) == float(sum(Fraction(float(x)) for x in v))
