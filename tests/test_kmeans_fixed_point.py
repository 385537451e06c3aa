"""The fixed-point member sums of the GPU k-means (FP32 rows).

Every entry is rounded to round(x 2^q) and the integers are added exactly;
q = 62 - E - L with max |x| < 2^E and n <= 2^L.  These tests restate that
rule and the conversion the kernel uses (an FP32 value above 2^23 is an
integer: its mantissa shifted left by exponent - 150; below, round to
nearest even in FP32) and check, with exact Python integers and fractions,
that the conversion is round-half-even, that no sum can pass 2^63, and that
a mean is within 2^-q of the exact mean of the FP32 rows."""
from fractions import Fraction
import math

import numpy as np
import pytest


def scale_exponent(xmax: float, n: int) -> int:
    E = math.frexp(xmax)[1] if xmax > 0 else 0  # xmax < 2^E (frexp: m in [0.5, 1))
    L = 0
    while L < 62 and (1 << L) < n:
        L += 1
    return 62 - E - L


def fixed(y: np.float32) -> int:
    """The kernel's conversion of an FP32 y, |y| < 2^62, to an integer."""
    if abs(float(y)) < 8388608.0:
        return int(np.rint(np.float32(y)))  # FP32 round to nearest even
    b = int(np.array(y, dtype=np.float32).view(np.uint32))
    v = ((b & 0x7FFFFF) | 0x800000) << (((b >> 23) & 0xFF) - 150)
    return -v if b >> 31 else v


def round_half_even(y: np.float32) -> int:
    f = Fraction(float(y))
    fl = math.floor(f)
    r = f - fl
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and fl % 2 == 1):
        return fl + 1
    return fl


def test_conversion_is_round_half_even():
    rng = np.random.default_rng(0)
    ys = []
    for e in range(-3, 62):
        ys += list((rng.uniform(1, 2, 40) * 2.0 ** e) * rng.choice([-1, 1], 40))
    ys += [0.5, 1.5, 2.5, -0.5, -2.5, 8388607.5, 8388608.0, -8388609.0, 2.0 ** 61 * 1.75]
    for y in ys:
        y32 = np.float32(y)
        if abs(float(y32)) >= 2.0 ** 62:
            continue
        assert fixed(y32) == round_half_even(y32), y


@pytest.mark.parametrize("n,xmax", [(1, 1.0), (1000, 0.06), (4097, 3.0e5), (1 << 20, 1e-20), (3, 1e30)])
def test_no_sum_can_overflow(n, xmax):
    q = scale_exponent(xmax, n)
    per_entry = Fraction(xmax) * Fraction(2) ** q + Fraction(1, 2)  # |round(x 2^q)| bound
    assert n * per_entry < 2 ** 63


@pytest.mark.parametrize("seed", range(4))
def test_mean_within_two_to_minus_q(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 3000))
    mag = 10.0 ** rng.uniform(-8, 8)
    x = (rng.standard_normal(n) * mag).astype(np.float32)
    q = scale_exponent(float(np.max(np.abs(x))), n)
    assert -120 <= q <= 120  # the kernel's scale 2^q is a normal FP32 number
    scale = np.float32(2.0 ** q)
    total = sum(fixed(np.float32(v) * scale) for v in x)  # x 2^q is exact in FP32
    assert abs(total) < 2 ** 62 + n
    exact = sum(Fraction(float(v)) for v in x) / n
    got = Fraction(total, n) / Fraction(2) ** q
    assert abs(got - exact) <= Fraction(1, 2) / Fraction(2) ** q
