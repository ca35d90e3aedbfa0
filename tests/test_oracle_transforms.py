"""Pins of the oracle's exact transforms (Background: Algorithms 1.2, 2.2, 3, 4, 5).

Each transform must satisfy its defining identity EXACTLY in rational
arithmetic (a+b = s+t, a-b = d+t, ab = p+e, a = qb+r, a = c^2+d) away from
underflow and overflow, and its main result must be the plain IEEE result
(checked with Python's own float operations, independent of the oracle)."""
import math

import numpy as np
import pytest

import oracle as O
from tests.fp import F, rand_doubles, same

N = 4000


def make_pairs():
    rng = np.random.default_rng(1234)
    a = rand_doubles(rng, N, -40, 40)
    b = rand_doubles(rng, N, -40, 40)
    # edge bands: equal / opposite magnitudes, powers of two, zeros, close values
    extra_a = [1.0, 1.0, -1.0, 0.0, -0.0, 2.0 ** 52, 1.5, 3.0, 1e300, 1e-300, 0.1, 0.1]
    extra_b = [1.0, -1.0, 2.0 ** -53, 0.0, 0.0, 0.5, -1.5, -2.9999999999999996, 1e300, -1e-300,
               0.2, -0.09999999999999999]
    return np.concatenate([a, extra_a]), np.concatenate([b, extra_b])


@pytest.fixture(scope="module")
def pairs():
    return make_pairs()


def test_two_sum_exact(pairs):
    a, b = pairs
    for x, y in zip(a, b):
        s, t = O.two_sum(x, y)
        assert same(s, x + y)
        assert F(x) + F(y) == F(s) + F(t), (x, y, s, t)


def test_two_diff_exact(pairs):
    """Two-Diff with the sign reading of steps (4),(5): a - b = d + t exactly."""
    a, b = pairs
    for x, y in zip(a, b):
        d, t = O.two_diff(x, y)
        assert same(d, x - y)
        assert F(x) - F(y) == F(d) + F(t), (x, y, d, t)


def test_two_diff_as_printed_would_fail():
    """The printed order b# = b - b', a# = a' - a yields -t: the pin above
    would catch it (checked here on one case with a nonzero error)."""
    a, b = 1.0, 2.0 ** -60
    d = a - b
    b1 = a - d
    a1 = b1 + d
    t_printed = (b - b1) + (a1 - a)
    _, t = O.two_diff(a, b)
    assert t != 0 and t_printed == -t
    assert F(a) - F(b) != F(d) + F(t_printed)


def test_two_prod_exact(pairs):
    a, b = pairs
    for x, y in zip(a, b):
        p, e = O.two_prod(x, y)
        assert same(p, x * y)
        if x != 0 and y != 0 and not (2.0 ** -960 < abs(p) < 2.0 ** 1000):
            continue                      # outside the band where e is exact
        assert F(x) * F(y) == F(p) + F(e), (x, y)


def test_div_rem_exact(pairs):
    a, b = pairs
    for x, y in zip(a, b):
        if y == 0:
            continue
        q, r = O.div_rem(x, y)
        assert same(q, x / y)
        if x != 0 and not (2.0 ** -960 < abs(q) < 2.0 ** 1000):
            continue
        assert F(x) == F(q) * F(y) + F(r), (x, y)


def test_sqrt_rem_exact(pairs):
    a, _ = pairs
    for x in np.abs(a):
        c, d = O.sqrt_rem(x)
        assert same(c, math.sqrt(x))
        if x != 0 and not (2.0 ** -900 < x < 2.0 ** 1000):
            continue
        assert F(x) == F(c) * F(c) + F(d), x


def test_zero_error_is_positive_zero():
    """Exact results carry a +0 error (round-to-nearest: x - x = +0)."""
    for fn, args in ((O.two_sum, (1.0, 2.0)), (O.two_diff, (3.0, 1.0)), (O.two_prod, (3.0, 0.5)),
                     (O.two_sum, (5.0, -0.0)), (O.two_diff, (-0.0, 0.0)),
                     (O.div_rem, (1.0, 4.0))):
        hi, lo = fn(*args)
        assert lo == 0.0 and math.copysign(1.0, lo) == 1.0, (fn, args, lo)


def test_special_values_propagate():
    """No special casing (Algorithms, Methodic): Inf and NaN flow through."""
    s, t = O.two_sum(math.inf, 1.0)
    assert s == math.inf and math.isnan(t)
    s, t = O.two_sum(1e308, 1e308)          # overflow of the sum
    assert s == math.inf and math.isnan(t)
    p, e = O.two_prod(math.nan, 1.0)
    assert math.isnan(p) and math.isnan(e)
    q, r = O.div_rem(1.0, 0.0)
    assert q == math.inf and math.isnan(r)
    c, d = O.sqrt_rem(-1.0)
    assert math.isnan(c) and math.isnan(d)
