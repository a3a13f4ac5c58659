"""Error bound of the float-float stencil sums of the FP32 criteria.

The FP32 path evaluates the Table 1 stencils (Sec. 2.2) on float-float
values with Dekker's sloppy addition, whose error is bounded in absolute
terms (about 2^-47 of the operands), and keeps the pairs unnormalised
inside a stencil.  This test restates those operations in float32 numpy
(round-to-nearest; a fused multiply-add formed from the exact double
product) and checks, against exact rational arithmetic on the same
float-float inputs, that the unnormalised chain stays within the sloppy
bound and within a small factor of the normalised chain's error, on data
with the cancellation of a smooth density (differences ~1e-4 of values ~1).
"""
from fractions import Fraction

import numpy as np

F = np.float32


def fma(a, b, c):
    # a*b is exact in double for float32 a, b; the sum rounds once to double
    # and once to float32 (the double rounding does not matter for a bound)
    return F(np.float64(a) * np.float64(b) + np.float64(c))


def two_sum(a, b):
    s = F(a + b)
    bb = F(s - a)
    return s, F(F(a - F(s - bb)) + F(b - bb))


def fast_two_sum(a, b):
    s = F(a + b)
    return s, F(b - F(s - a))


def add_abs(a, b):
    s, e = two_sum(a[0], b[0])
    return fast_two_sum(s, F(e + F(a[1] + b[1])))


def sub_abs(a, b):
    return add_abs(a, (F(-b[0]), F(-b[1])))


def add_raw(a, b):
    s, e = two_sum(a[0], b[0])
    return s, F(e + F(a[1] + b[1]))


def sub_raw(a, b):
    return add_raw(a, (F(-b[0]), F(-b[1])))


def mul_f_raw(a, k):
    ch = F(a[0] * k)
    return ch, fma(a[1], k, fma(a[0], k, -ch))


def mul_f(a, k):
    return fast_two_sum(*mul_f_raw(a, k))


def exact(a):
    return Fraction(float(a[0])) + Fraction(float(a[1]))


def to_ff(x):
    hi = F(x)
    return hi, F(x - np.float64(hi))


def d3_normalised(f):
    e = [sub_abs(f[3 + k], f[3 - k]) for k in (1, 2, 3)]
    return sub_abs(add_abs(mul_f(e[0], F(-13)), mul_f(e[1], F(8))), e[2])


def d3_unnormalised(f):
    e = [sub_raw(f[3 + k], f[3 - k]) for k in (1, 2, 3)]
    return sub_abs(add_raw(mul_f_raw(e[0], F(-13)), mul_f_raw(e[1], F(8))), e[2])


def d2_normalised(f):
    s = [add_abs(f[3 + k], f[3 - k]) for k in (1, 2, 3)]
    return add_abs(add_abs(mul_f(s[0], F(270)), mul_f(s[1], F(-27))),
                   add_abs(mul_f(s[2], F(2)), mul_f(f[3], F(-490))))


def d2_unnormalised(f):
    s = [add_raw(f[3 + k], f[3 - k]) for k in (1, 2, 3)]
    return add_abs(add_raw(mul_f_raw(s[0], F(270)), mul_f_raw(s[1], F(-27))),
                   add_raw(mul_f_raw(s[2], F(2)), mul_f_raw(f[3], F(-490))))


def _exact_d3(f):
    x = [exact(v) for v in f]
    return -13 * (x[4] - x[2]) + 8 * (x[5] - x[1]) - (x[6] - x[0])


def _exact_d2(f):
    x = [exact(v) for v in f]
    return 270 * (x[4] + x[2]) - 27 * (x[5] + x[1]) + 2 * (x[6] + x[0]) - 490 * x[3]


def test_unnormalised_stencil_sums_keep_the_sloppy_bound():
    rng = np.random.default_rng(20251113)
    worst = {"d3n": 0.0, "d3u": 0.0, "d2n": 0.0, "d2u": 0.0}
    for _ in range(400):
        # seven consecutive values of a smooth density near 1 (the stencil's
        # inputs cancel to ~1e-4) with float-float representations
        x0, slope, curv = 1.0 + rng.uniform(-0.3, 0.3), rng.uniform(-1, 1) * 1e-4, rng.uniform(-1, 1) * 1e-7
        f = [to_ff(x0 + slope * k + curv * k * k + rng.uniform(-1, 1) * 1e-12) for k in range(-3, 4)]
        scale = max(abs(float(v[0])) for v in f)
        for name, fn, ex in (("d3n", d3_normalised, _exact_d3), ("d3u", d3_unnormalised, _exact_d3),
                             ("d2n", d2_normalised, _exact_d2), ("d2u", d2_unnormalised, _exact_d2)):
            err = abs(float(exact(fn(f)) - ex(f))) / scale
            worst[name] = max(worst[name], err)
    # the sloppy bound: 2^-47 of the operands at each addition, so over a
    # stencil about 2^-46 times the sum of |weight| over its operands (each
    # weight but the centre's applies to two values): D3 2 (13 + 8 + 1) = 44,
    # D2 2 (270 + 27 + 2) + 490 = 1088
    bound = {"d3": 2.0 ** -46 * 44, "d2": 2.0 ** -46 * 1088}
    for name, err in worst.items():
        assert err <= bound[name[:2]], (name, err / 2.0 ** -47, bound[name[:2]] / 2.0 ** -47)
    # the unnormalised chains are no worse than a small factor of the
    # normalised ones
    assert worst["d3u"] <= 4 * max(worst["d3n"], 2.0 ** -52), worst
    assert worst["d2u"] <= 4 * max(worst["d2n"], 2.0 ** -52), worst


def test_a_dropped_low_part_breaks_the_bound():
    """The bound is tight enough to see a mistake: losing the low parts (the
    stencil in plain float) misses it by orders of magnitude."""
    rng = np.random.default_rng(7)
    worst = 0.0
    for _ in range(100):
        x0, slope = 1.0 + rng.uniform(-0.3, 0.3), rng.uniform(-1, 1) * 1e-4
        f = [to_ff(x0 + slope * k + rng.uniform(-1, 1) * 1e-12) for k in range(-3, 4)]
        g = [(v[0], F(0)) for v in f]  # low parts dropped
        err = abs(float(exact(d3_unnormalised(g)) - _exact_d3(f))) / max(abs(float(v[0])) for v in f)
        worst = max(worst, err)
    assert worst > 1e3 * 2.0 ** -46 * 44
