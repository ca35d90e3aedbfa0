"""Pins of the oracle's twofold algorithms (Algorithms section).

* strictness claims: ATF/STF 1.1 and DTF 1.1.1 return z1 = RN(dz0) exactly,
  MTF 1.1 with x1 = 0 returns the exact product error;
* special-case reductions stated in the paper (DTF 1.1 with x1 = 0 is
  DTF 1.1.1; RTF 1 with x1 = 0 is RPF 1.1 in value; MTF 1 with zero tails is
  Two-Product);
* the worked examples of the Add/subtract, Divide and Root sections;
* rounding-error budgets of the general algorithms derived from their exact
  expansions (dz0 = x1 + y1 + e for ATF1, e00 + x0y1 + x1y0 + x1y1 for MTF1,
  (x - z0 y)/y for DTF1, the first-order root correction of RTF1 with its
  exact remainder term), with tails spread over the epsilon-order regimes so
  that a dropped term, a wrong sign or a swapped operand exceeds the budget.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from tests.fp import EPS, F, U, fma, isqrt_frac, rand_doubles, rand_tails, rn, same, ulp

N = 3000


def make_data():
    rng = np.random.default_rng(99)
    x0 = rand_doubles(rng, N, -30, 30)
    y0 = rand_doubles(rng, N, -30, 30)
    x1 = rand_tails(rng, x0, 0, 70)
    y1 = rand_tails(rng, y0, 0, 70)
    return x0, x1, y0, y1


@pytest.fixture(scope="module")
def data():
    return make_data()


# ----------------------------------------------------------- strict variants

def test_atf11_strict(data):
    x0, x1, y0, _ = data
    for a0, a1, b0 in zip(x0, x1, y0):
        z0, z1 = O.atf11(a0, a1, b0)
        assert same(z0, a0 + b0)
        dz0 = F(a0) + F(a1) + F(b0) - F(z0)
        assert same(z1, rn(dz0)), (a0, a1, b0)


def test_stf11_strict(data):
    x0, x1, y0, _ = data
    for a0, a1, b0 in zip(x0, x1, y0):
        z0, z1 = O.stf11(a0, a1, b0)
        assert same(z0, a0 - b0)
        dz0 = F(a0) + F(a1) - F(b0) - F(z0)
        assert same(z1, rn(dz0)), (a0, a1, b0)


def test_mtf11_dotted_is_two_prod(data):
    x0, _, y0, _ = data
    for a0, b0 in zip(x0, y0):
        z0, z1 = O.mtf11(a0, 0.0, b0)
        assert same(z0, a0 * b0)
        assert F(z1) == F(a0) * F(b0) - F(z0)


def test_dtf111_strict(data):
    """Divide: Q1 = q0 + q1 is the best 2x-precise quotient, q1 = RN(a/b - q0)."""
    x0, _, y0, _ = data
    for a0, b0 in zip(x0, y0):
        z0, z1 = O.dtf111(a0, b0)
        assert same(z0, a0 / b0)
        assert same(z1, rn(F(a0) / F(b0) - F(z0))), (a0, b0)


def test_dtf11_reduces_to_dtf111(data):
    x0, _, y0, _ = data
    for a0, b0 in zip(x0, y0):
        assert all(same(u, v) for u, v in zip(O.dtf11(a0, 0.0, b0), O.dtf111(a0, b0)))


def test_rtf1_x1_zero_is_rpf11_in_value(data):
    x0, _, _, _ = data
    for a0 in np.abs(x0):
        z = O.rtf1(a0, 0.0)
        w = O.rpf11(a0)
        assert same(z[0], w[0]) and z[1] == w[1], a0


def test_rpf11_output_coupled(data):
    """RPF 1.1 output is non-overlapping: |z1| <= ulp(z0)/2, and z1 is the
    Newton correction of a correctly rounded sqrt: within 2u|z1| of dz0."""
    x0, _, _, _ = data
    for a0 in np.abs(x0):
        z0, z1 = O.rpf11(a0)
        assert same(z0, math.sqrt(a0))
        assert abs(z1) <= ulp(z0) / 2
        dz0 = isqrt_frac(F(a0)) - F(z0)
        assert abs(F(z1) - dz0) <= 4 * U * abs(F(z1)) + F(z0) * U * U * 4


def test_mtf1_zero_tails_is_two_prod(data):
    """Dotted inputs given as twofolds with +0 tails: MTF1 returns the exact
    product error bit for bit (e00 (+) +0 (+) (+-0 (+) +-0) = e00)."""
    x0, _, y0, _ = data
    for a0, b0 in zip(x0, y0):
        z = O.mtf1(a0, 0.0, b0, 0.0)
        p, e = O.two_prod(a0, b0)
        assert same(z[0], p) and same(z[1], e)


# ----------------------------------------------------------- worked examples

def test_example_atf1_miss():
    """Add/subtract: x = 1 - eps, y = eps - eps^2 -> z0 = 1, z1 = 0 while the
    exact dz0 = -eps^2 (a documented miss of the fast algorithm)."""
    z0, z1 = O.atf1(1.0, -EPS, EPS, -EPS * EPS)
    assert z0 == 1.0 and z1 == 0.0
    exact = F(1.0) - F(EPS) + F(EPS) - F(EPS) ** 2 - F(z0)
    assert exact == -Fraction(1, 2 ** 106)


def test_example_dtf1():
    """Divide: x = (1, 0), y = (1 - eps, eps): z0 = 1 + 2 eps,
    r0 = -eps + 2 eps^2, r1 = -eps - 2 eps^2, z1 = c0 = -2 eps = dz0 exactly."""
    x0, x1, y0, y1 = 1.0, 0.0, 1.0 - EPS, EPS
    z0, z1 = O.dtf1(x0, x1, y0, y1)
    assert z0 == 1.0 + 2 * EPS
    q, r0 = O.div_rem(x0, y0)
    assert F(r0) == -F(EPS) + 2 * F(EPS) ** 2
    r1 = fma(-z0, y1, x1)
    assert F(r1) == -F(EPS) - 2 * F(EPS) ** 2
    assert z1 == -2 * EPS
    assert F(z1) == (F(x0) + F(x1)) / (F(y0) + F(y1)) - F(z0)


def test_example_rtf1():
    """Root: x0 = x1 = 1: z0 = 1, u = (2, 0), z0 + z1 ~ sqrt(2)."""
    z0, z1 = O.rtf1(1.0, 1.0)
    assert z0 == 1.0
    assert O.two_sum(1.0, 1.0) == (2.0, 0.0)
    r2 = isqrt_frac(Fraction(2))
    assert abs(F(z0) + F(z1) - r2) <= 2 * F(ulp(z1))


def test_dtf111_corner_cases():
    """Divide by zero gives Inf/NaN and NaN propagates (Divide section)."""
    z0, z1 = O.dtf111(1.0, 0.0)
    assert z0 == math.inf and math.isnan(z1)
    z0, z1 = O.dtf111(0.0, 0.0)
    assert math.isnan(z0) and math.isnan(z1)
    z0, z1 = O.dtf111(math.nan, 2.0)
    assert math.isnan(z0) and math.isnan(z1)


def test_rpf_domain():
    """Root: a negative argument raises the domain error (NaN)."""
    z0, z1 = O.rpf11(-4.0)
    assert math.isnan(z0) and math.isnan(z1)
    z0, z1 = O.rtf1(-4.0, 1e-20)
    assert math.isnan(z0) and math.isnan(z1)


def test_sqrt_zero_literal_nan():
    """sqrt(+0) through RPF 1.1 divides 0 by 2*0: z1 is NaN (no special case)."""
    z0, z1 = O.rpf11(0.0)
    assert z0 == 0.0 and math.isnan(z1)


# ------------------------------------------------ budgets of the general ops

def _budget_ok(err, budget):
    return abs(err) <= budget * (1 + Fraction(1, 2 ** 40)) + Fraction(1, 2 ** 1070)


def test_atf1_budget(data):
    """dz0 = x1 + y1 + e exactly; z1 = RN(RN(x1 + y1) + e): two roundings."""
    x0, x1, y0, y1 = data
    for a0, a1, b0, b1 in zip(x0, x1, y0, y1):
        z0, z1 = O.atf1(a0, a1, b0, b1)
        assert same(z0, a0 + b0)
        dz0 = F(a0) + F(a1) + F(b0) + F(b1) - F(z0)
        u = a1 + b1
        assert _budget_ok(F(z1) - dz0, U * (abs(F(u)) + abs(F(z1)))), (a0, a1, b0, b1)


def test_stf1_budget(data):
    x0, x1, y0, y1 = data
    for a0, a1, b0, b1 in zip(x0, x1, y0, y1):
        z0, z1 = O.stf1(a0, a1, b0, b1)
        assert same(z0, a0 - b0)
        dz0 = F(a0) + F(a1) - F(b0) - F(b1) - F(z0)
        u = a1 - b1
        assert _budget_ok(F(z1) - dz0, U * (abs(F(u)) + abs(F(z1)))), (a0, a1, b0, b1)


def test_mtf1_budget(data):
    """dz0 = e00 + x0 y1 + x1 y0 + x1 y1 exactly; the fast formula rounds the
    three products and three sums."""
    x0, x1, y0, y1 = data
    for a0, a1, b0, b1 in zip(x0, x1, y0, y1):
        z0, z1 = O.mtf1(a0, a1, b0, b1)
        assert same(z0, a0 * b0)
        dz0 = (F(a0) + F(a1)) * (F(b0) + F(b1)) - F(z0)
        p00, e00 = O.two_prod(a0, b0)
        p11, p01, p10 = a1 * b1, a0 * b1, a1 * b0
        s1, s2 = e00 + p11, p01 + p10
        budget = U * (abs(F(p11)) + abs(F(p01)) + abs(F(p10)) + abs(F(s1)) + abs(F(s2)) + abs(F(z1)))
        assert _budget_ok(F(z1) - dz0, budget), (a0, a1, b0, b1)


def test_dtf1_budget(data):
    """x - z0 y = r0 + (x1 - z0 y1) with r0 exact; z1 = RN(RN(r0 + RN(x1 - z0 y1)) / RN(y0 + y1)).
    Budget: the two roundings of the remainder, the rounding of the
    denominator and of the final quotient (the Divide section's ~3 eps|q1|)."""
    x0, x1, y0, y1 = data
    for a0, a1, b0, b1 in zip(x0, x1, y0, y1):
        z0, z1 = O.dtf1(a0, a1, b0, b1)
        assert same(z0, a0 / b0)
        y = F(b0) + F(b1)
        dz0 = (F(a0) + F(a1)) / y - F(z0)
        _, r0 = O.div_rem(a0, b0)
        r1 = fma(-z0, b1, a1)
        c0 = r0 + r1
        d0 = b0 + b1
        q = F(c0) / F(d0)
        budget = (U * abs(F(z1)) + abs(q) * abs(y - F(d0)) / abs(y)
                  + U * (abs(F(r1)) + abs(F(c0))) / abs(y))
        assert _budget_ok(F(z1) - dz0, budget), (a0, a1, b0, b1)


def test_dtf11_budget(data):
    x0, x1, y0, _ = data
    for a0, a1, b0 in zip(x0, x1, y0):
        z0, z1 = O.dtf11(a0, a1, b0)
        dz0 = (F(a0) + F(a1)) / F(b0) - F(z0)
        _, r = O.div_rem(a0, b0)
        c = r + a1
        budget = U * abs(F(z1)) + U * abs(F(c)) / abs(F(b0))
        assert _budget_ok(F(z1) - dz0, budget), (a0, a1, b0)


def test_rtf1_coupled_loose(data):
    """Coupled input (|x1| below half an ulp of x0): z0 + z1 is close to the
    exact root, |dz1| <= 8 u^2 |z0| + 2 u |z1|."""
    x0, _, _, _ = data
    rng = np.random.default_rng(5)
    a0s = np.abs(x0)
    a1s = (rng.random(a0s.size) - 0.5) * np.array([ulp(v) for v in a0s])
    for a0, a1 in zip(a0s, a1s):
        z0, z1 = O.rtf1(a0, a1)
        assert same(z0, math.sqrt(a0))
        exact = isqrt_frac(F(a0) + F(a1))
        err = F(z0) + F(z1) - exact
        assert abs(err) <= 8 * U * U * F(z0) + 2 * U * abs(F(z1)), (a0, a1)


def rtf1_inputs():
    """x0 > 0 with tails of every size: coupled (below half an ulp), spread
    over the epsilon-order regimes, up to half of x0 and up to nine times
    it (where v0 and z0 are more than a factor 2 apart and Two-Diff's tail
    is not zero)."""
    rng = np.random.default_rng(7)
    a0 = np.abs(rand_doubles(rng, 4000, -30, 30))
    a1 = np.concatenate([(rng.random(1000) - 0.5) * np.array([ulp(v) for v in a0[:1000]]),
                         rand_tails(rng, a0[1000:2000], 1, 70),
                         a0[2000:3000] * (rng.random(1000) - 0.5),
                         a0[3000:] * rng.uniform(-0.9, 9.0, 1000)])
    return a0, a1


def test_rtf1_budget():
    """The Root section's RTF1 step by step, each rounding bounded (u = 2^-53,
    |RN(a) - a| <= u |RN(a)|):
      z0 = RN(sqrt x0);  (u0, u1) = Two-Sum(x0, x1), so u0 + u1 = x0 + x1 = X;
      RPF1: v0 = RN(sqrt u0), d = u0 - v0^2 exactly (Algorithm 5),
            c = RN(u1 + d), v1 = RN(c / (2 v0));
      STF1.1: w0 = RN(v0 - z0) with the exact tail e, w1 = RN(v1 + e);
      z1 = RN(w0 + w1).
    With delta = u1 + d = X - v0^2 and s = sqrt(X), the identity
    s - v0 - delta/(2 v0) = -delta^2 / (2 v0 (s + v0)^2) gives
      z0 + z1 - s = delta^2/(2 v0 (s + v0)^2) + rho_c/(2 v0) + rho_v1 + rho_w1 + rho_z1,
    so |z0 + z1 - s| <= delta^2/(2 v0 (s + v0)^2) + u |c|/(2 v0) + u (|v1| + |w1| + |z1|).
    Checked against the exact root of the exact input (300 bits)."""
    a0s, a1s = rtf1_inputs()
    for a0, a1 in zip(a0s, a1s):
        z0, z1 = O.rtf1(a0, a1)
        assert same(z0, math.sqrt(a0))
        X = F(a0) + F(a1)
        s = isqrt_frac(X)
        u0, u1 = O.two_sum(a0, a1)
        v0 = math.sqrt(u0)
        d = fma(-v0, v0, u0)
        c = u1 + d
        v1 = c / (2.0 * v0)
        w0, e = O.two_diff(v0, z0)
        w1 = v1 + e
        delta = X - F(v0) * F(v0)
        model = delta * delta / (2 * F(v0) * (s + F(v0)) ** 2)
        budget = model + U * (abs(F(c)) / (2 * F(v0)) + abs(F(v1)) + abs(F(w1)) + abs(F(z1)))
        err = F(z0) + F(z1) - s
        assert abs(err) <= budget * (1 + Fraction(1, 2 ** 40)) + s * Fraction(1, 2 ** 290), (a0, a1, float(err))


# --------------------------------------------------------------- panic flag

def test_flag_rel_and_nonfinite():
    tau = 2.0 ** -40
    assert O.flag(1.0, 2.0 ** -41) == 0
    assert O.flag(1.0, 2.0 ** -40) == 0            # strict inequality
    assert O.flag(1.0, -2.0 ** -39) == O.PANIC
    assert O.flag(0.0, 0.0) == 0
    assert O.flag(0.0, 1e-300) == O.PANIC
    assert O.flag(math.nan, 1.0) == O.NONFINITE      # NaN compares false
    assert O.flag(1.0, math.inf) == O.NONFINITE | O.PANIC
    assert O.flag(math.inf, math.nan) == O.NONFINITE
    assert O.flag(3.0, 3.0 * tau * 1.0000001, O.REL, tau) == O.PANIC


def test_flag_ulp_mode():
    for z0 in (1.0, 3.5, 1e-300, 2.0 ** -1074, 0.0, 1e300):
        u = ulp(z0)
        assert O.flag(z0, 4 * u, O.ULP, 0.0, 4.0) == 0
        assert O.flag(z0, math.nextafter(4 * u, math.inf), O.ULP, 0.0, 4.0) == O.PANIC


def test_flag_rel_threshold_in_ulps():
    """2^-40 |z0| lies in [2^12, 2^13) ulp(z0) for normal z0."""
    rng = np.random.default_rng(3)
    for z0 in rand_doubles(rng, 200, -300, 300):
        t = F(2.0 ** -40) * abs(F(z0)) / F(ulp(z0))
        assert 2 ** 12 <= t < 2 ** 13
