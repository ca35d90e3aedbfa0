"""Pins of the oracle's Horner evaluation and elementwise programs.

Horner: z0 equals plain Horner written here with Python floats; the
coefficients of (x-1)^k are exact binomials (C(30,15) < 2^53) and x - 1 is
exact for x in [0.9, 1.1] (Sterbenz), so p(x) is known exactly and z0 + z1
must meet the compensated-Horner bound gamma_2k^2 * p~(|x|) (Graillat,
Langlois, Louvet 2005).

Elementwise chain z = sqrt((a*b + c)/d): z0 equals numpy's plain
evaluation (no contraction) bit for bit; z0 + z1 approaches the exact root
of the exact twofold inputs far beyond binary64 precision.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle as O
import synth
from tests.fp import bits, canon, isqrt_frac, rand_doubles, rand_tails

u = 2.0 ** -53


def gamma(n):
    return n * u / (1 - n * u)


def horner_py(a, x):
    s = float(a[-1])
    for c in reversed(a[:-1]):
        t = s * x
        s = t + float(c)
    return s


@pytest.mark.parametrize("k", [0, 1, 5, 10, 20, 30])
def test_horner_binomial(k):
    a = synth.binomial_coefs(k)
    assert all(float(v).is_integer() and abs(v) < 2 ** 53 for v in a)
    x = synth.horner_points(400, seed=3)
    z0, z1, fl = O.horner(a, x)
    zp = O.horner_plain(a, x)
    for i, xv in enumerate(x):
        ref = horner_py(a, float(xv))
        assert bits(z0[i]) == bits(ref) and bits(zp[i]) == bits(ref)
        exact = (Fr(float(xv)) - 1) ** k
        ptilde = (1 + abs(Fr(float(xv)))) ** k
        err = abs(Fr(z0[i]) + Fr(z1[i]) - exact)
        assert err <= Fr(gamma(2 * k + 2) ** 2) * ptilde * 2, (k, xv)
        assert fl[i] == O.flag(z0[i], z1[i])


def test_horner_panic_grows_with_degree():
    x = synth.horner_points(2000, seed=4)
    rates = []
    for k in (1, 5, 10, 20, 30):
        z0, z1, fl = O.horner(synth.binomial_coefs(k), x)
        rates.append(np.mean(fl & O.PANIC))
    assert rates[0] == 0.0
    assert all(b >= a for a, b in zip(rates, rates[1:]))
    assert rates[-1] > 0.99


CHAIN = [(O.MUL, 4, 0, 1), (O.ADD, 5, 4, 2), (O.DIV, 6, 5, 3), (O.SQRT, 7, 6, 6)]


def chain_inputs(n, seed=0):
    d = synth.ew_chain(n, seed)
    return [(d["a0"], d["a1"]), (d["b0"], d["b1"]), (d["c0"], d["c1"]), (d["d0"], d["d1"])]


def test_chain_z0_is_plain_numpy():
    ins = chain_inputs(20000)
    z0, z1, fl = O.ew(CHAIN, ins)
    a, b, c, d = (h for h, _ in ins)
    with np.errstate(invalid="ignore"):
        ref = np.sqrt((a * b + c) / d)
    assert np.array_equal(canon(z0), canon(ref))
    assert np.array_equal(canon(O.ew_plain(CHAIN, [h for h, _ in ins])), canon(ref))
    nan = np.isnan(ref)
    assert 0.4 < nan.mean() < 0.6                      # half the radicands are negative
    assert np.all(fl[nan] == O.NONFINITE) and np.all(np.isnan(z1[nan]))


def test_chain_tail_tracks_exact_error():
    ins = chain_inputs(600, seed=2)
    z0, z1, _ = O.ew(CHAIN, ins)
    (a0, a1), (b0, b1), (c0, c1), (d0, d1) = ins
    checked = 0
    for i in range(600):
        if math.isnan(z0[i]):
            continue
        A = Fr(a0[i]) + Fr(a1[i])
        B = Fr(b0[i]) + Fr(b1[i])
        C = Fr(c0[i]) + Fr(c1[i])
        D = Fr(d0[i]) + Fr(d1[i])
        rad = (A * B + C) / D
        if rad <= 0:
            continue
        exact = isqrt_frac(rad)
        kappa = (abs(A * B) + abs(C)) / abs(A * B + C)
        err = abs(Fr(z0[i]) + Fr(z1[i]) - exact)
        assert err <= Fr(2.0 ** -95) * exact * (1 + kappa), i
        checked += 1
    assert checked > 200


def test_program_kinds_against_scalar_ops():
    """The interpreter dispatches the operand kinds like the scalar op entry,
    and its z0 equals the plain evaluation of the program."""
    rng = np.random.default_rng(7)
    n = 300
    x0 = rand_doubles(rng, n, -5, 5)
    x1 = rand_tails(rng, x0, 40, 60)
    y0 = np.abs(rand_doubles(rng, n, -5, 5))
    w0 = rand_doubles(rng, n, -5, 5)
    prog = [(O.SUB, 3, 0, 1), (O.MUL, 4, 2, 3), (O.DIV, 5, 4, 1), (O.ADD, 6, 5, 2),
            (O.SQRT, 7, 1, 1), (O.MUL, 8, 6, 7)]
    ins = [(x0, x1), (y0, None), (w0, None)]
    z0, z1, fl = O.ew(prog, ins)
    for i in range(n):
        r3 = O.op(O.SUB, (x0[i], x1[i]), y0[i])
        r4 = O.op(O.MUL, w0[i], r3)
        r5 = O.op(O.DIV, r4, y0[i])
        r6 = O.op(O.ADD, r5, w0[i])
        r7 = O.op(O.SQRT, y0[i])
        r8 = O.op(O.MUL, r6, r7)
        assert bits(z0[i]) == bits(r8[0]) and bits(z1[i]) == bits(r8[1])
        plain = (w0[i] * (x0[i] - y0[i]) / y0[i] + w0[i]) * math.sqrt(y0[i])
        assert bits(z0[i]) == bits(plain)
