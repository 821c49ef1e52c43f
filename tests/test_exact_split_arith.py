"""The error-free transformations behind the FP64-grade residual on the FP32 pipe, replayed on the host with
the same bit operations and float32 roundings (numpy), against exact rational arithmetic:

- the three-float split of a double (a = a1 + a2 + a3 exactly, a1 the 24-bit truncation, a2 the next 24 bits,
  a3 the last 5), built from the exponent and fraction bits and integer-to-float conversions;
- the three-level sum of products (Knuth two-sums for the leading and the next-order level, the FMA two-product
  for the product errors), whose error must stay far below an FP64 accumulation's.
"""
from fractions import Fraction

import numpy as np

F32 = np.float32


def _bits_to_f32(b):
    return np.array([b & 0xFFFFFFFF], dtype=np.uint32).view(np.float32)[0]


def _f32_bits(x):
    return int(np.array([x], dtype=np.float32).view(np.uint32)[0])


def split3(a):
    """The split as the device code does it, with Python integers for the bit fields."""
    u = int(np.array([a], dtype=np.float64).view(np.uint64)[0])
    uh, ul = u >> 32, u & 0xFFFFFFFF
    e = (uh >> 20) & 0x7FF
    if e < 1023 - 60 or e > 1023 + 100:
        a1 = F32(a)
        r = a - float(a1)
        a2 = F32(r)
        return a1, a2, F32(r - float(a2))
    sign = uh & 0x80000000
    frac23 = ((uh << 3) | (ul >> 29)) & 0x007FFFFF
    a1 = _bits_to_f32(sign | ((e - 1023 + 127) << 23) | frac23)
    rem = ul & 0x1FFFFFFF
    top, low = rem >> 5, rem & 31
    a2 = _bits_to_f32(sign | (_f32_bits(F32(top)) + ((e - 1070) << 23))) if top else F32(0.0)
    a3 = _bits_to_f32(sign | (_f32_bits(F32(low)) + ((e - 1075) << 23))) if low else F32(0.0)
    return a1, a2, a3


def two_sum(a, b):
    s = F32(a + b)
    v = F32(s - a)
    return s, F32(F32(a - F32(s - v)) + F32(b - v))


def fma32(a, b, c):
    # float32 operands: a * b is exact in FP64 (48 bits); the uses below are exact in float32 as well
    return F32(float(a) * float(b) + float(c))


class XAcc:
    def __init__(self):
        self.h = self.m = self.l = F32(0.0)

    def add_prod(self, a1, a2, a3, x):
        p1 = F32(a1 * x)
        e1 = fma32(a1, x, -p1)
        p2 = F32(a2 * x)
        e2 = fma32(a2, x, -p2)
        p3 = F32(a3 * x)
        self.h, t0 = two_sum(self.h, p1)
        s, u1 = two_sum(self.m, t0)
        m, u2 = two_sum(s, e1)
        self.m, u3 = two_sum(m, p2)
        self.l = F32(self.l + F32(F32(u1 + u2) + F32(u3 + F32(e2 + p3))))

    def value(self):
        return (float(self.l) + float(self.m)) + float(self.h)


def test_three_float_split_is_exact():
    rng = np.random.default_rng(5)
    vals = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.uniform(-15, 25, 4000),
                           [0.0, -0.0, 1.0, -1.0, 2.0 ** -60, 2.0 ** 99, 1e-30, 2.0 ** 120, np.pi, -np.e]])
    for a in vals:
        a = float(a)
        a1, a2, a3 = split3(a)
        assert Fraction(a) == Fraction(float(a1)) + Fraction(float(a2)) + Fraction(float(a3)), a
        if 2.0 ** -60 <= abs(a) < 2.0 ** 100:
            assert abs(float(a2)) <= 2.0 ** -23 * abs(a) and abs(float(a3)) <= 2.0 ** -47 * abs(a)


def test_three_level_sum_of_products_beats_fp64():
    """Residual-like sums with heavy cancellation: sum_j a_j x_j - g with a FP64, x float32; the three-level
    sum's error against exact arithmetic stays below 2^-60 of sum |a_j x_j|, well under the FP64 FMA
    accumulation's (about N 2^-53 at worst, measured here too)."""
    rng = np.random.default_rng(7)
    worst = worst64 = 0.0
    for trial in range(6):
        n = 300
        a = rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n))
        x = rng.standard_normal(n).astype(np.float32)
        x[-1] = np.float32(-(np.dot(a[:-1], x[:-1].astype(np.float64)) / a[-1]))   # near-cancelling sum
        exact = sum(Fraction(float(ai)) * Fraction(float(xi)) for ai, xi in zip(a, x))
        acc = XAcc()
        s64 = 0.0
        for ai, xi in zip(a, x):
            acc.add_prod(*split3(float(ai)), xi)
            s64 = float(np.fma(ai, float(xi), s64)) if hasattr(np, "fma") else s64 + ai * float(xi)
        scale = float(sum(abs(Fraction(float(ai)) * Fraction(float(xi))) for ai, xi in zip(a, x)))
        worst = max(worst, abs(float(Fraction(acc.value()) - exact)) / scale)
        worst64 = max(worst64, abs(float(Fraction(s64) - exact)) / scale)
    assert worst < 2.0 ** -60, worst
    assert worst < worst64 or worst64 == 0.0
