"""Pins of the binary32 basis of the oracle: exact transforms and strict
variants against exact rational arithmetic rounded to binary32, the float
rows of the paper's application logs (tests/golden/paper_logs.txt: gauss
well3 / ill3, test100h, quadratic, and the float conversions of their
inputs), the renormalising accumulator of the Applications section in the
paper's own binary24 format, the sticky flag, and rounding-error budgets of
the general add, subtract, multiply, divide and root derived from their
steps (the binary64 tests' derivations with u = 2^-24)."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from tests.fp import F, U32, f32, isqrt_frac, rn32, split32, ulp32
from tests.test_oracle_applications import g6, golden


def rand32(rng, n, emin=-20, emax=20):
    m = rng.integers(1 << 23, 1 << 24, n).astype(np.float64)
    e = rng.integers(emin, emax + 1, n) - 23
    s = np.where(rng.integers(0, 2, n) == 1, -1.0, 1.0)
    return (s * np.ldexp(m, e)).astype(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def pairs():
    rng = np.random.default_rng(32)
    return rand32(rng, 20000), rand32(rng, 20000)


def test_rn32_helper():
    """The binary32 rounding of the tests agrees with numpy's on doubles
    (which are exact rationals) and rounds ties to even."""
    rng = np.random.default_rng(0)
    for v in rng.standard_normal(2000) * 10.0 ** rng.integers(-30, 30, 2000):
        assert rn32(F(v)) == f32(v)
    assert rn32(Fraction(1) + Fraction(1, 2 ** 24)) == 1.0            # tie -> even
    assert rn32(Fraction(1) + Fraction(3, 2 ** 24)) == 1.0 + 2.0 ** -22


def test_exact_transforms32(pairs):
    a, b = pairs
    for x, y in zip(a, b):
        s, t = O.two_sum32(x, y)
        assert s == rn32(F(x) + F(y)) and F(s) + F(t) == F(x) + F(y)
        d, t = O.two_diff32(x, y)
        assert d == rn32(F(x) - F(y)) and F(d) + F(t) == F(x) - F(y)
        p, e = O.two_prod32(x, y)
        assert p == rn32(F(x) * F(y))
        if abs(p) > 2.0 ** -100:
            assert F(p) + F(e) == F(x) * F(y)
        q, r = O.div_rem32(x, y)
        assert q == rn32(F(x) / F(y))
        if abs(x) > 2.0 ** -80:
            assert F(q) * F(y) + F(r) == F(x)
        c, dd = O.sqrt_rem32(abs(x))
        assert F(c) ** 2 + F(dd) == abs(F(x))


def test_strict_variants32(pairs):
    """ATF 1.1, STF 1.1 and MTF 1.1 of a dotted tail: z1 = RN32(exact dz0)."""
    a, b = pairs
    rng = np.random.default_rng(5)
    for x0, y0 in zip(a, b):
        x1 = f32(x0 * 2.0 ** -int(rng.integers(10, 30)) * rng.uniform(-1, 1))
        z0, z1 = O.op32(O.ADD, (x0, x1), y0)
        assert z1 == rn32(F(x0) + F(x1) + F(y0) - F(z0))
        z0, z1 = O.op32(O.SUB, (x0, x1), y0)
        assert z1 == rn32(F(x0) + F(x1) - F(y0) - F(z0))
        z0, z1 = O.op32(O.MUL, x0, y0)             # Two-Product
        assert z1 == rn32(F(x0) * F(y0) - F(z0))


def test_atf1_stf1_budget32(pairs):
    """General twofold add / subtract: dz0 = x1 +- y1 + e exactly, z1 rounds
    twice (RN32(RN32(x1 +- y1) + e)): |z1 - dz0| <= u (|x1 +- y1| + |z1|)."""
    a, b = pairs
    rng = np.random.default_rng(8)
    for x0, y0 in zip(a, b):
        x1 = f32(x0 * 2.0 ** -int(rng.integers(5, 30)) * rng.uniform(-1, 1))
        y1 = f32(y0 * 2.0 ** -int(rng.integers(5, 30)) * rng.uniform(-1, 1))
        for code, sg in ((O.ADD, 1), (O.SUB, -1)):
            z0, z1 = O.op32(code, (x0, x1), (y0, y1))
            dz0 = F(x0) + F(x1) + sg * (F(y0) + F(y1)) - F(z0)
            u = f32(x1 + sg * y1)
            budget = U32 * (abs(F(u)) + abs(F(z1)))
            assert abs(F(z1) - dz0) <= budget * (1 + Fraction(1, 2 ** 20)) + Fraction(1, 2 ** 149), (code, x0, x1, y0, y1)


def test_dtf111_and_rpf11_32(pairs):
    """DTF 1.1.1: z1 = RN32(r / y) with r the exact remainder; RPF 1.1 output
    coupled and within 4 u |z1| of the exact root's error."""
    a, b = pairs
    for x, y in zip(a, b):
        z0, z1 = O.op32(O.DIV, x, y)
        _, r = O.div_rem32(x, y)
        assert z1 == rn32(F(r) / F(y))
        c0, c1 = O.op32(O.SQRT, abs(x))
        assert abs(c1) <= ulp32(c0) / 2
        dz0 = isqrt_frac(abs(F(x))) - F(c0)
        assert abs(F(c1) - dz0) <= 4 * U32 * abs(F(c1)) + F(c0) * U32 * U32 * 4


def _tailed(rng, heads, kmin, kmax):
    """binary32 tails |x1| ~ |x0| 2^-k, k uniform in [kmin, kmax]."""
    return np.array([f32(h * 2.0 ** -int(rng.integers(kmin, kmax + 1)) * rng.uniform(-1, 1)) for h in heads])


def _ok32(err, budget):
    return abs(err) <= budget * (1 + Fraction(1, 2 ** 20)) + Fraction(1, 2 ** 149)


def test_mtf1_budget32(pairs):
    """General twofold multiply: dz0 = e00 + x0 y1 + x1 y0 + x1 y1 exactly;
    the formula rounds the three products and three sums once each."""
    a, b = (v[:6000] for v in pairs)
    rng = np.random.default_rng(10)
    x1s, y1s = _tailed(rng, a, 1, 30), _tailed(rng, b, 1, 30)
    for x0, x1, y0, y1 in zip(a, x1s, b, y1s):
        z0, z1 = O.op32(O.MUL, (x0, x1), (y0, y1))
        assert z0 == rn32(F(x0) * F(y0))
        dz0 = (F(x0) + F(x1)) * (F(y0) + F(y1)) - F(z0)
        _, e00 = O.two_prod32(x0, y0)
        p11, p01, p10 = rn32(F(x1) * F(y1)), rn32(F(x0) * F(y1)), rn32(F(x1) * F(y0))
        s1, s2 = rn32(F(e00) + F(p11)), rn32(F(p01) + F(p10))
        budget = U32 * sum(abs(F(v)) for v in (p11, p01, p10, s1, s2, z1))
        assert _ok32(F(z1) - dz0, budget), (x0, x1, y0, y1)


def test_dtf1_budget32(pairs):
    """General twofold divide: x - z0 y = r0 + (x1 - z0 y1) with r0 exact;
    z1 = RN(RN(r0 + RN(x1 - z0 y1)) / RN(y0 + y1)).  Budget: the rounding of
    the remainder's two terms, of the denominator and of the quotient."""
    a, b = (v[:6000] for v in pairs)
    rng = np.random.default_rng(11)
    x1s, y1s = _tailed(rng, a, 1, 30), _tailed(rng, b, 1, 30)
    for x0, x1, y0, y1 in zip(a, x1s, b, y1s):
        z0, z1 = O.op32(O.DIV, (x0, x1), (y0, y1))
        assert z0 == rn32(F(x0) / F(y0))
        y = F(y0) + F(y1)
        dz0 = (F(x0) + F(x1)) / y - F(z0)
        _, r0 = O.div_rem32(x0, y0)
        r1 = rn32(F(x1) - F(z0) * F(y1))
        c0, d0 = rn32(F(r0) + F(r1)), rn32(F(y0) + F(y1))
        q = F(c0) / F(d0)
        budget = U32 * abs(F(z1)) + abs(q) * abs(y - F(d0)) / abs(y) + U32 * (abs(F(r1)) + abs(F(c0))) / abs(y)
        assert _ok32(F(z1) - dz0, budget), (x0, x1, y0, y1)


def test_rtf1_budget32(pairs):
    """Twofold root, its steps in binary32 with the binary64 test's
    derivation: Two-Sum (exact), RPF1 on (u0, u1) with the exact residual d
    and the exact remainder delta^2 / (2 v0 (s + v0)^2) of the first-order
    correction (delta = u1 + d), STF1.1 against z0, one rounding per step;
    tails from below half an ulp to nine times x0."""
    a = np.abs(pairs[0][:6000])
    rng = np.random.default_rng(12)
    x1s = np.concatenate([_tailed(rng, a[:2000], 25, 40), _tailed(rng, a[2000:4000], 1, 24),
                          np.array([f32(h * rng.uniform(-0.9, 9.0)) for h in a[4000:]])])
    for x0, x1 in zip(a, x1s):
        z0, z1 = O.op32(O.SQRT, (x0, x1))
        assert z0 == rn32(isqrt_frac(F(x0), 80))
        X = F(x0) + F(x1)
        s = isqrt_frac(X)
        u0, u1 = O.two_sum32(x0, x1)
        v0, d = O.sqrt_rem32(u0)
        c = rn32(F(u1) + F(d))
        v1 = rn32(F(c) / (2 * F(v0)))
        _, e = O.two_diff32(v0, z0)
        w1 = rn32(F(v1) + F(e))
        delta = X - F(v0) * F(v0)
        model = delta * delta / (2 * F(v0) * (s + F(v0)) ** 2)
        budget = model + U32 * (abs(F(c)) / (2 * F(v0)) + abs(F(v1)) + abs(F(w1)) + abs(F(z1)))
        err = F(z0) + F(z1) - s
        assert _ok32(err, budget), (x0, x1, float(err), float(budget))


# --------------------------------------------------------------- paper logs

def test_float_inputs_as_printed():
    rows = golden()
    for v in ("0.1", "0.001", "1e-08"):
        h, t = split32(float(v))
        assert (g6(h), g6(t)) == rows[("f32_input", v)]


def T32(v):
    return (f32(v), 0.0)


@pytest.mark.parametrize("case,lam,f", [("gauss_well3_f32", 0.1, (11.0, 11.0, 1.0)),
                                        ("gauss_ill3_f32", 0.001, (1001.0, 1001.0, 1.0))])
def test_gauss_float_logs(case, lam, f):
    """Back substitution with the float twofold lambda of the log's matrix:
    all six printed digits of every head and tail."""
    rows = golden()
    L = split32(lam)
    x2 = O.op32(O.DIV, T32(f[2]), L)
    x1 = O.op32(O.DIV, O.op32(O.SUB, T32(f[1]), O.op32(O.MUL, T32(1.0), x2)), L)
    x0 = O.op32(O.DIV, O.op32(O.SUB, T32(f[0]), O.op32(O.MUL, T32(1.0), x1)), L)
    for i, (z0, z1) in enumerate((x0, x1, x2)):
        assert (g6(z0), g6(z1)) == rows[(case, str(i))], (case, i, z0, z1)


@pytest.mark.parametrize("h", [100, 1000])
def test_test100h_float_logs(h):
    """A sequential float twofold counter of the tick 0.1[-1.49012e-09],
    3600 x 10 ticks per hour, converted to hours by DTF 1.1: the printed
    96.3958[3.54008] and 582.542[461.249]."""
    n = h * 3600 * 10
    t0, t1 = split32(0.1)
    s = O.reduce_sum32(np.full(n, t0, np.float32), np.full(n, t1, np.float32), L=n)
    z0, z1 = O.op32(O.DIV, s, 3600.0)
    assert (g6(z0), g6(z1)) == golden()[("test100h_f32", str(h))]


def quadratic32(c):
    a, b = T32(1.0), T32(2.0)
    cc = split32(c)
    bb = O.op32(O.MUL, b, b)
    ac4 = O.op32(O.MUL, O.op32(O.MUL, T32(4.0), a), cc)
    d = O.op32(O.SQRT, O.op32(O.SUB, bb, ac4))
    two_a = O.op32(O.MUL, T32(2.0), a)
    x0 = O.op32(O.DIV, O.op32(O.SUB, T32(-2.0), d), two_a)
    x1 = O.op32(O.DIV, O.op32(O.ADD, T32(-2.0), d), two_a)
    return d, x0, x1


def test_quadratic_float_logs_out_of_range():
    """c just above 1: the negative discriminant gives the printed heads
    0, -1, -1 with NaN tails."""
    rows = golden()
    d, x0, x1 = quadratic32(1 + 1e-8)
    for name, v in (("quadratic_f32_d", d), ("quadratic_f32_x0", x0), ("quadratic_f32_x1", x1)):
        assert (g6(v[0]), g6(v[1])) == rows[(name, "1.00000001")], (name, v)


def test_quadratic_float_logs_in_range():
    """x^2 + 2x + c, c = 1e-08, over float twofolds.  The log prints
    d = 2[1e-08], x0 = -2[-5e-09], x1 = 0[5e-09]: the heads and the tails'
    digits match, and the tails' signs are the opposite of the exact errors
    (d = sqrt(4 - 4c) < 2, so d's error is negative).  The same computation
    with Algorithm 2.2's printed signs (which return -t, see R1) reproduces
    the printed row exactly, so the log carries that sign slip; the exact
    Two-Diff gives the tails with the right signs, checked here against the
    exact root."""
    rows = golden()
    d, x0, x1 = quadratic32(1e-8)
    for name, v in (("quadratic_f32_d", d), ("quadratic_f32_x0", x0), ("quadratic_f32_x1", x1)):
        p0, p1 = rows[(name, "1e-08")]
        assert g6(v[0]) == p0 and g6(-v[1]) == p1, (name, v)
    c = F(split32(1e-8)[0]) + F(split32(1e-8)[1])
    exact_d = isqrt_frac(4 - 4 * c)
    assert exact_d - F(d[0]) < 0 and d[1] < 0
    assert abs(F(d[1]) - (exact_d - F(d[0]))) <= abs(exact_d - F(d[0])) * Fraction(1, 1000)
    d_p, t_p = O.two_diff32(4.0, f32(4e-8))
    assert F(d_p) + F(t_p) == 4 - F(f32(4e-8))       # the exact transform (R1)


def test_renormalising_accumulator_binary24():
    """Applications, in the paper's own format: adding unity to a binary32
    twofold accumulator saturates at z0 = z1 = 2^24 without renormalising
    and stays exact with it (from 2^25 - 1000, 3000 additions)."""
    z0, z1 = 2.0 ** 24, 2.0 ** 24 - 1000
    for _ in range(3000):
        z0, z1 = O.op32(O.ADD, (z0, z1), 1.0)
    assert (z0, z1) == (2.0 ** 24, 2.0 ** 24)
    p = O.op32(O.PADD, (2.0 ** 24, 2.0 ** 24 - 1000), 0.0)
    assert p == (2.0 ** 25 - 1000, 0.0)
    for _ in range(3000):
        p = O.op32(O.PADD, p, 1.0)
    assert p == (2.0 ** 25 + 2000, 0.0)


# --------------------------------------------------------------- sticky flag

def test_sticky_flag_keeps_an_intermediate_panic():
    """R12: (1 + tiny) - 1 = (0, tiny) panics (|z1| > tau |z0| = 0); times a
    dotted 0 gives (0, 0) and plus 1 gives (1, 0), both calm.  Only the
    sticky flag still reports the panic at the end, in both bases."""
    prog = [(O.SUB, 3, 0, 1), (O.MUL, 4, 3, 2), (O.ADD, 5, 4, 1)]
    ones, zero = np.ones(4), np.zeros(4)
    ins = [(np.ones(4), np.full(4, 2.0 ** -60)), (ones, None), (zero, None)]
    z0, z1, fl = O.ew(prog[:1], ins)
    assert (z0[0], z1[0]) == (0.0, 2.0 ** -60) and fl[0] == O.PANIC
    z0, z1, fl = O.ew(prog, ins, mode=O.REL)
    assert (z0[0], z1[0]) == (1.0, 0.0) and list(fl) == [0] * 4
    z0, z1, fl = O.ew(prog, ins, mode=O.REL | O.STICKY)
    assert (z0[0], z1[0]) == (1.0, 0.0) and list(fl) == [O.PANIC] * 4
    ins32 = [(np.ones(4, np.float32), np.full(4, 2.0 ** -30, np.float32)), (ones, None), (zero, None)]
    assert list(O.ew32(prog, ins32, mode=O.REL)[2]) == [0] * 4
    assert list(O.ew32(prog, ins32, mode=O.REL | O.STICKY)[2]) == [O.PANIC] * 4


# ------------------------------------------------ binary32 sum and dot (R8)

def test_dot32_single_term_is_two_product(pairs):
    """A one-element dotted dot is the Two-Product pair: z0 + z1 = x y
    exactly, z0 = RN(x y)."""
    x, y = pairs
    for a, b in zip(x[:500], y[:500]):
        z0, z1 = O.reduce32([a], None, [b])
        assert F(z0) + F(z1) == F(a) * F(b)
        assert z0 == rn32(F(a) * F(b))


def test_dot32_with_unit_multiplier_is_the_sum():
    """y = 1: every Two-Product is (x, +0), and ATF1 with a +0 tail adds the
    same bits as ATF1.1, so the dot equals the dotted sum bit for bit."""
    rng = np.random.default_rng(5)
    for n, L in [(1, 256), (255, 256), (1000, 7), (5000, 256), (777, 1000)]:
        x = rand32(rng, n, -10, 10).astype(np.float32)
        d = O.reduce32(x, None, np.ones(n, np.float32), L=L)
        s = O.reduce_sum32(x, None, L=L)
        assert np.array_equal(np.float32(d).view(np.uint32), np.float32(s).view(np.uint32)), (n, L)


def test_dot32_zero_tails_equal_dotted():
    """Materialised +0 tails give the dotted result (MTF1.1 with x1 = 0
    adds 0 y0 = +-0 to the Two-Product tail, which keeps it)."""
    rng = np.random.default_rng(6)
    n = 3000
    x = rand32(rng, n).astype(np.float32)
    y = rand32(rng, n).astype(np.float32)
    z = np.zeros(n, np.float32)
    a = O.reduce32(x, None, y, None)
    for xl, yl in [(z, None), (None, z), (z, z)]:
        b = O.reduce32(x, xl, y, yl)
        assert np.array_equal(np.float32(a).view(np.uint32), np.float32(b).view(np.uint32))


def test_dot32_exact_when_everything_is_representable():
    """Small integers: every product and partial sum is exact in binary32,
    so z0 is the exact dot and z1 = 0, for any leaf size."""
    rng = np.random.default_rng(7)
    for n, L in [(10, 3), (1000, 256), (4096, 64), (999, 1)]:
        x = rng.integers(-60, 61, n).astype(np.float32)
        y = rng.integers(-60, 61, n).astype(np.float32)
        z0, z1 = O.reduce32(x, None, y, None, L=L)
        assert z0 == float(np.dot(x.astype(np.int64), y.astype(np.int64))) and z1 == 0.0


def test_dot32_accuracy_and_z0_is_the_plain_dot():
    """z0 is the plain binary32 dot in the same order (each step's head is the
    rounded plain operation), and z0 + z1 is within the twofold error bound
    of the exact dot: |err| <= u |dot| + 2 n^2 u^2 sum |x_i y_i| (u = 2^-24),
    which plain binary32 accumulation misses by orders of magnitude on
    cancelling data."""
    rng = np.random.default_rng(8)
    u = Fraction(1, 2 ** 24)
    for n, L in [(50, 256), (700, 64), (2000, 256)]:
        for trial in range(5):
            x = rand32(rng, n, -8, 8).astype(np.float32)
            y = rand32(rng, n, -8, 8).astype(np.float32)
            z0, z1 = O.reduce32(x, None, y, None, L=L)
            plain = O.reduce32_plain(x, y, L=L)
            assert np.float32(z0).view(np.uint32) == np.float32(plain).view(np.uint32)
            exact = sum(F(float(a)) * F(float(b)) for a, b in zip(x, y))
            mag = sum(abs(F(float(a)) * F(float(b))) for a, b in zip(x, y))
            assert abs(F(z0) + F(z1) - exact) <= u * abs(exact) + 2 * n * n * u * u * mag


def test_plain32_twin_is_plain_float_arithmetic():
    """The plain twin is binary32 IEEE arithmetic in the blocked order:
    numpy float32 operations in the same order give the same bits."""
    rng = np.random.default_rng(9)
    for n, L in [(1, 4), (100, 7), (1000, 256), (257, 256)]:
        x = rand32(rng, n).astype(np.float32)
        y = rand32(rng, n).astype(np.float32)
        for dot in (False, True):
            nodes = []
            for j in range(0, n, L):
                s = np.float32(0.0)
                for i in range(j, min(n, j + L)):
                    s = np.float32(s + (np.float32(x[i] * y[i]) if dot else x[i]))
                nodes.append(s)
            while len(nodes) > 1:
                nodes = [np.float32(nodes[i] + nodes[i + 1]) for i in range(0, len(nodes) - 1, 2)] + \
                        ([nodes[-1]] if len(nodes) % 2 else [])
            got = O.reduce32_plain(x, y if dot else None, L=L)
            assert np.float32(got).view(np.uint32) == nodes[0].view(np.uint32), (n, L, dot)
