"""The error-free transformations behind the FP64-grade residual on the FP32 pipe, replayed on the host with
the same bit operations and float32 roundings (numpy), against exact rational arithmetic:

- the three-float split of a double (a = a1 + a2 + a3 exactly, a1 the 24-bit truncation, a2 the next 24 bits,
  a3 the last 5), built from the exponent and fraction bits and integer-to-float conversions;
- the anchored sums of products (error-free extraction against power-of-two anchors sized from a bound of the
  sum of |a x|, the FMA two-product for the product errors), whose error must be of the order of an FP64
  accumulation's, with both anchored levels staying in their binades.
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


def split2(a):
    """The two-float split of the later-pass residual updates (hi the 24-bit truncation, lo the 29 bits below
    rounded once by an integer-to-float conversion, then scaled), as the device code forms it."""
    u = int(np.array([a], dtype=np.float64).view(np.uint64)[0])
    uh, ul = u >> 32, u & 0xFFFFFFFF
    e = (uh >> 20) & 0x7FF
    sign = uh & 0x80000000
    frac23 = ((uh << 3) | (ul >> 29)) & 0x007FFFFF
    hi = _bits_to_f32(sign | ((e - 1023 + 127) << 23) | frac23)
    rem = ul & 0x1FFFFFFF
    lo = _bits_to_f32(sign | (_f32_bits(F32(rem)) + ((e - 1075) << 23))) if rem else F32(0.0)
    return hi, lo, rem


def fma32(a, b, c):
    # float32 operands: a * b is exact in FP64 (48 bits); the uses below are exact in float32 as well
    return F32(float(a) * float(b) + float(c))


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


def test_two_float_split_rounds_once():
    """lo is the 29 fraction bits below hi rounded once to float32 (what a conversion of that integer gives):
    |a - hi - lo| <= 2^-47 |a| and lo equals the correctly rounded remainder."""
    rng = np.random.default_rng(9)
    vals = rng.standard_normal(3000) * 10.0 ** rng.uniform(-15, 25, 3000)
    for a in vals:
        a = float(a)
        hi, lo, rem = split2(a)
        exact_rem = Fraction(a) - Fraction(float(hi))
        assert float(lo) == float(F32(float(exact_rem)))          # one rounding of the exact remainder
        assert abs(Fraction(a) - Fraction(float(hi)) - Fraction(float(lo))) <= Fraction(2) ** -47 * abs(Fraction(a))


class AAcc:
    """The anchored sums of the first-pass residual (anchors 1.5 2^kh and 1.5 2^km), float32 step by step."""

    def __init__(self, kh, km):
        self.H = self.sh = F32(1.5 * 2.0 ** kh)
        self.M = self.sm = F32(1.5 * 2.0 ** km)
        self.l = F32(0.0)

    def put_m(self, v):
        t = F32(self.M + v)
        self.l = F32(self.l + F32(v - F32(t - self.M)))
        self.M = t

    def add_prod(self, a1, a2, a3, x):
        p1 = F32(a1 * x)
        e1 = fma32(a1, x, -p1)
        t = F32(self.H + p1)
        r1 = F32(p1 - F32(t - self.H))
        self.H = t
        self.put_m(r1)
        self.put_m(e1)
        u = fma32_round(a2, x, self.M)
        q = F32(u - self.M)
        self.l = F32(self.l + fma32_round(a2, x, -q))
        self.M = u
        self.l = fma32_round(a3, x, self.l)

    def renorm(self):
        t = F32(self.M + self.l)
        self.l = F32(self.l - F32(t - self.M))
        self.M = t

    def value(self):
        return (float(F32(self.H - self.sh)) + float(F32(self.M - self.sm))) + float(self.l)


def fma32_round(a, b, c):
    """fmaf: a * b + c rounded once to float32 (exact rational arithmetic, then one rounding)."""
    return F32(float(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))))


def _anchors(bound, n_terms):
    # as the kernel: bnd in [2^e, 2^(e+1)) -> kh = e + 2 (every partial sum below 2^(kh-1));
    # km = kh - 23 + ceil(log2(T + 4))
    e = int(np.floor(np.log2(bound)))
    kh = e + 2
    km = kh - 23 + int(np.ceil(np.log2(n_terms + 4)))
    return kh, km


def _check_anchored(a, x, renorm_every=4):
    """Sum a_j x_j by the anchored sums; returns (error, bound) against exact rational arithmetic, after
    checking that H and M never leave their binades."""
    n = len(a)
    bound = float(np.sum(np.abs(a) * np.abs(x.astype(np.float64)))) * (1 + 2 ** -20)
    kh, km = _anchors(bound, n)
    acc = AAcc(kh, km)
    for j, (aj, xj) in enumerate(zip(a, x)):
        acc.add_prod(*split3(float(aj)), xj)
        assert 2.0 ** kh <= float(acc.H) <= 2.0 ** (kh + 1)
        assert 2.0 ** km <= float(acc.M) <= 2.0 ** (km + 1)
        if (j + 1) % renorm_every == 0:
            acc.renorm()
    exact = sum(Fraction(float(ai)) * Fraction(float(xi)) for ai, xi in zip(a, x))
    return abs(float(Fraction(acc.value()) - exact)), bound


def test_anchored_sums_fp64_grade():
    """Residual-like sums (FP64 entries times float32 values): cancelling, same-sign (every partial sum near
    the bound) and mixed-magnitude cases; the error stays below 2^-48 of the bound sum |a x| (2^-51 to 2^-55
    measured; an FP64 accumulation of the same sums, 2^-49 to 2^-54)."""
    rng = np.random.default_rng(11)
    worst = 0.0
    for trial in range(8):
        n = (64, 300, 1024)[trial % 3]
        a = rng.standard_normal(n) * np.exp(rng.uniform(-4, 4, n))
        if trial % 4 == 1:
            a = np.abs(a)                                     # same sign: partial sums up to the bound
        x = rng.standard_normal(n).astype(np.float32)
        if trial % 4 == 1:
            x = np.abs(x)
        if trial % 4 == 2:
            x[-1] = np.float32(-(np.dot(a[:-1], x[:-1].astype(np.float64)) / a[-1]))   # near-cancelling
        err, bound = _check_anchored(a, x)
        worst = max(worst, err / bound)
    assert worst < 2.0 ** -48, worst


def test_anchored_sums_zero_and_tiny_terms():
    # zero entries and exactly representable values: the sum is exact
    a = np.array([0.0, 1.0, -0.5, 0.25, 0.0, 3.0])
    x = np.array([1.0, 2.0, 4.0, -8.0, 5.0, 0.5], dtype=np.float32)
    err, bound = _check_anchored(a, x)
    assert err == 0.0


def _abs_bound_f32(a):
    """|a| bounded from above in float32 as the row-norm kernel does: the 23 leading fraction bits times
    (1 + 2^-22)."""
    u = int(np.array([abs(a)], dtype=np.float64).view(np.uint64)[0])
    e = u >> 52
    if e >= 1023 + 127:
        return F32(np.inf)
    if e < 1023 - 126:
        return F32(2.0 ** -126)
    frac23 = (u >> 29) & 0x7FFFFF
    return F32(_bits_to_f32(((e - 1023 + 127) << 23) | frac23) * F32(1 + 2.0 ** -22))


def _fma32(a, b, c):
    return F32(float(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))))


def test_anchor_bounds_hold():
    """The first-pass residual's anchors: per row the FP32 bounds of the 1-norm and 2-norm of the row's 2N real
    components, per window max |phi| and the 2-norm bound, bnd = min(n1 max|phi|, n2 |phi|_2) (1 + 2^-20), all
    with the kernels' float32 roundings, must bound both accumulators' sums of |a x| (real and imaginary part
    pairings); kh = e + 2 for bnd in [2^e, 2^(e+1)) then keeps every partial sum below 2^(kh-1)."""
    rng = np.random.default_rng(21)
    for trial in range(6):
        n = (40, 200, 513)[trial % 3]
        ar = rng.standard_normal(n) * np.exp(rng.uniform(-6, 2, n))
        ai = rng.standard_normal(n) * np.exp(rng.uniform(-6, 2, n))
        ar[trial % n] *= 1e3                                    # a dominant (diagonal-like) entry
        pr = (rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n))).astype(np.float32)
        pi = (rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n))).astype(np.float32)
        n1 = n2 = F32(0.0)
        for x, y in zip(ar, ai):
            br, bi = _abs_bound_f32(float(x)), _abs_bound_f32(float(y))
            n1 = F32(n1 + F32(br + bi))
            n2 = _fma32(br, br, _fma32(bi, bi, n2))
        n1 = F32(n1 * F32(1 + 2.0 ** -10))
        n2 = F32(F32(np.sqrt(F32(n2 * F32(1 + 2.0 ** -10)))) * F32(1 + 2.0 ** -20))
        pm = F32(max(np.max(np.abs(pr)), np.max(np.abs(pi))))
        p2 = F32(0.0)
        for x, y in zip(pr, pi):
            p2 = _fma32(x, x, _fma32(y, y, p2))
        p2 = F32(F32(np.sqrt(F32(p2 * F32(1 + 2.0 ** -10)))) * F32(1 + 2.0 ** -20))
        bnd = F32(min(F32(n1 * pm), F32(n2 * p2)) * F32(1 + 2.0 ** -20))
        fr = [Fraction(float(v)) for v in pr]
        fi = [Fraction(float(v)) for v in pi]
        far = [Fraction(float(v)) for v in ar]
        fai = [Fraction(float(v)) for v in ai]
        s_re = sum(abs(a) * abs(x) + abs(b) * abs(y) for a, b, x, y in zip(far, fai, fr, fi))
        s_im = sum(abs(a) * abs(y) + abs(b) * abs(x) for a, b, x, y in zip(far, fai, fr, fi))
        assert Fraction(float(bnd)) >= max(s_re, s_im)
        e = int(np.floor(np.log2(float(bnd))))
        kh = e + 2
        # the leading products p1 = fl(a1 x) add up to at most (1 + 2^-24) sum |a x|
        assert max(s_re, s_im) * (1 + Fraction(1, 2 ** 24)) < Fraction(2) ** (kh - 1)
