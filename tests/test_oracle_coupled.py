"""Pins of the coupled ("p", Dekker emulation) operations of the oracle:
Fast Two-Sum (Algorithm 1.1) and its precondition, renormalised outputs that
are coupled and keep the pair's value, MPF 1 / DPF 1 / RPF 1 against the
exact result of coupled inputs (rounding budgets derived from the exact
expansions), the paper's renormalisation example (the saturating accumulator
of the Applications section, at binary64's saturation point), and the
reading that dotted-only operations need no renormalisation."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from tests.fp import F, U, fma, isqrt_frac, rand_doubles, same, ulp

N = 2000


def coupled_tails(rng, heads):
    """|x1| <= ulp(x0)/2: a non-overlapping ("coupled") twofold."""
    u = np.array([ulp(float(h)) for h in heads])
    return u / 2 * rng.uniform(-1, 1, heads.size)


def make_coupled(seed=7):
    rng = np.random.default_rng(seed)
    x0 = rand_doubles(rng, N, -30, 30)
    y0 = rand_doubles(rng, N, -30, 30)
    return x0, coupled_tails(rng, x0), y0, coupled_tails(rng, y0)


@pytest.fixture(scope="module")
def cdata():
    return make_coupled()


def _ok(err, budget):
    return abs(err) <= budget * (1 + Fraction(1, 2 ** 40)) + Fraction(1, 2 ** 1070)


# -------------------------------------------------------------- Fast Two-Sum

def test_fast_two_sum_exact_when_ordered():
    """Algorithm 1.1: for |a| >= |b|, s = RN(a + b) and s + t = a + b exactly."""
    rng = np.random.default_rng(1)
    a = rand_doubles(rng, 20000, -40, 40)
    b = rand_doubles(rng, 20000, -40, 40)
    for x, y in zip(a, b):
        if abs(x) < abs(y):
            x, y = y, x
        s, t = O.fast_two_sum(x, y)
        assert same(s, x + y)
        assert F(s) + F(t) == F(x) + F(y), (x, y)


def test_fast_two_sum_needs_the_order():
    """With |a| < |b| the three operations lose the error: a = 2^-60, b = 1
    gives t = 0 while a + b - s = 2^-60 (hence its use for renormalising only
    a pair whose head dominates)."""
    s, t = O.fast_two_sum(2.0 ** -60, 1.0)
    assert s == 1.0 and t == 0.0
    assert F(2.0 ** -60) + 1 - F(s) == Fraction(1, 2 ** 60)


# -------------------------------------------------------- renormalised output

OPS = [(O.PADD, "add"), (O.PSUB, "sub"), (O.PMUL, "mul"), (O.PDIV, "div")]


@pytest.mark.parametrize("code,name", OPS)
@pytest.mark.parametrize("kinds", ["tt", "td", "dt"])
def test_coupled_outputs_are_coupled(cdata, code, name, kinds):
    """A p-operation of coupled operands returns a non-overlapping pair:
    |z1| <= ulp(z0)/2."""
    x0, x1, y0, y1 = cdata
    for a0, a1, b0, b1 in zip(x0, x1, y0, y1):
        x = (a0, a1) if kinds[0] == "t" else a0
        y = (b0, b1) if kinds[1] == "t" else b0
        z0, z1 = O.op(code, x, y)
        assert abs(z1) <= ulp(z0) / 2, (name, kinds, a0, a1, b0, b1, z0, z1)


def test_renormalisation_keeps_the_value(cdata):
    """Renormalising a head-dominated pair changes its split, not its value:
    the p-result sums exactly to the unrenormalised fast result."""
    x0, x1, y0, y1 = cdata
    for a0, a1, b0, b1 in zip(x0, x1, y0, y1):
        for fast, code in ((O.atf1(a0, a1, b0, b1), O.PADD), (O.stf1(a0, a1, b0, b1), O.PSUB),
                           (O.mpf1(a0, a1, b0, b1), O.PMUL), (O.dpf1(a0, a1, b0, b1), O.PDIV)):
            if abs(fast[0]) < abs(fast[1]) or not all(map(math.isfinite, fast)):
                continue
            z0, z1 = O.op(code, (a0, a1), (b0, b1))
            assert F(z0) + F(z1) == F(fast[0]) + F(fast[1]), (code, a0, a1, b0, b1)


def test_sqrt_coupled_output(cdata):
    x0, x1, _, _ = cdata
    for a0, a1 in zip(np.abs(x0), x1):
        z0, z1 = O.op(O.PSQRT, (a0, a1))
        assert abs(z1) <= ulp(z0) / 2


# ------------------------------------------------------- algorithms vs exact

def test_mpf1_budget(cdata):
    """dz0 = e00 + x0 y1 + x1 y0 + x1 y1 exactly; MPF 1 drops x1 y1 (minor for
    coupled input) and rounds p01, p10 and the two sums."""
    x0, x1, y0, y1 = cdata
    for a0, a1, b0, b1 in zip(x0, x1, y0, y1):
        z0, z1 = O.mpf1(a0, a1, b0, b1)
        assert same(z0, a0 * b0)
        dz0 = (F(a0) + F(a1)) * (F(b0) + F(b1)) - F(z0)
        p01, p10 = a0 * b1, a1 * b0
        budget = abs(F(a1) * F(b1)) + U * (abs(F(p01)) + abs(F(p10)) + abs(F(p01 + p10)) + abs(F(z1)))
        assert _ok(F(z1) - dz0, budget), (a0, a1, b0, b1)


def test_dpf1_budget(cdata):
    """dz0 = (r0 + (x1 - z0 y1)) / (y0 + y1) with r0 exact; DPF 1 divides by y0
    instead of y0 + y1 (relative |y1/y0| <= eps for coupled y) and rounds r1,
    c0 and the quotient."""
    x0, x1, y0, y1 = cdata
    for a0, a1, b0, b1 in zip(x0, x1, y0, y1):
        z0, z1 = O.dpf1(a0, a1, b0, b1)
        assert same(z0, a0 / b0)
        dz0 = (F(a0) + F(a1)) / (F(b0) + F(b1)) - F(z0)
        _, r0 = O.div_rem(a0, b0)
        r1 = fma(-z0, b1, a1)
        c0 = r0 + r1
        budget = (U * abs(F(r1)) + U * abs(F(c0))) / abs(F(b0)) + abs(dz0) * abs(F(b1) / F(b0)) + U * abs(F(z1))
        assert _ok(F(z1) - dz0, budget), (a0, a1, b0, b1)


def test_rpf1_budget(cdata):
    """For coupled x: dz0 = (x1 + d)/(2 z0 + dz0) with d = x0 - z0^2 exact;
    RPF 1 drops dz0 from the divisor and rounds the sum and the quotient."""
    x0, x1, _, _ = cdata
    for a0, a1 in zip(np.abs(x0), x1):
        z0, z1 = O.rpf1(a0, a1)
        assert same(z0, math.sqrt(a0))
        dz0 = isqrt_frac(F(a0) + F(a1)) - F(z0)
        c, d = O.sqrt_rem(a0)
        t = a1 + d
        budget = U * abs(F(t)) / (2 * F(z0)) + U * abs(F(z1)) + dz0 * dz0 / F(z0) + F(z0) * Fraction(1, 2 ** 250)
        assert _ok(F(z1) - dz0, budget), (a0, a1)


# ------------------------------------------------ the paper's renormalising example

def test_renormalising_accumulator_does_not_saturate():
    """Applications: adding unity to a twofold accumulator saturates without
    renormalising (in binary24 at z0 = z1 = 2^24) and stays exact with it.
    The same mechanism at binary64's saturation point: from 2^54 - 1000, add
    1.0 three thousand times."""
    z0, z1 = 2.0 ** 53, 2.0 ** 53 - 1000          # = 2^54 - 1000, head and tail both at 2^53
    for _ in range(3000):
        z0, z1 = O.op(O.ADD, (z0, z1), 1.0)
    assert (z0, z1) == (2.0 ** 53, 2.0 ** 53)      # saturated: the tail stopped growing
    p0, p1 = O.op(O.PADD, (2.0 ** 53, 2.0 ** 53 - 1000), 0.0)   # renormalised start
    assert (p0, p1) == (2.0 ** 54 - 1000, 0.0)
    for _ in range(3000):
        p0, p1 = O.op(O.PADD, (p0, p1), 1.0)
    assert F(p0) + F(p1) == 2 ** 54 + 2000
    assert (p0, p1) == (2.0 ** 54 + 2000, 0.0)


# ------------------------------------------------- R10: dotted needs no renormalising

def test_dotted_outputs_are_already_coupled():
    """With every operand dotted the exact transforms, DTF 1.1.1 and RPF 1.1
    already return non-overlapping pairs that Fast Two-Sum leaves unchanged,
    so returning them as is (R10) is the renormalised result too."""
    rng = np.random.default_rng(3)
    a = rand_doubles(rng, 20000, -60, 60)
    b = rand_doubles(rng, 20000, -60, 60)
    for x, y in zip(a, b):
        for code in (O.ADD, O.SUB, O.MUL, O.DIV):
            z = O.op(code, x, y)
            assert O.fast_two_sum(*z) == z, (code, x, y)
            assert O.op(code + 5, x, y) == z
        z = O.op(O.SQRT, abs(x))
        assert O.fast_two_sum(*z) == z
        assert O.op(O.PSQRT, abs(x)) == z
