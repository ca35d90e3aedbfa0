"""Exact-arithmetic helpers for the tests (binary64 facts from IEEE 754)."""
from __future__ import annotations

import math
import struct
from fractions import Fraction

import numpy as np

U = Fraction(1, 2 ** 53)          # unit roundoff of binary64, round to nearest
EPS = 2.0 ** -53                  # the paper's epsilon = ulp(1)/2


def F(x) -> Fraction:
    return Fraction(float(x))


def ulp(x: float) -> float:
    """Spacing of binary64 at x: 2^(max(e,-1022)-52)."""
    if x == 0 or not math.isfinite(x):
        return 2.0 ** -1074 if x == 0 else math.nan
    m, e = math.frexp(abs(x))     # x = m 2^e, m in [0.5, 1)
    return 2.0 ** (max(e - 1, -1022) - 52)


def rn(q: Fraction) -> float:
    """Round a rational to the nearest binary64 (ties to even): Python's
    Fraction.__float__ is correctly rounded."""
    return float(q)


def bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def same(a: float, b: float) -> bool:
    """Bitwise equality with every NaN treated as one value."""
    if math.isnan(a) or math.isnan(b):
        return math.isnan(a) and math.isnan(b)
    return bits(a) == bits(b)


def canon(a: np.ndarray) -> np.ndarray:
    """Bits of a float64 array with NaNs canonicalised (payloads differ across
    x86, arm64 and the GPU; that is the one allowed difference)."""
    a = np.ascontiguousarray(a, np.float64).copy()
    a[np.isnan(a)] = np.nan
    v = a.view(np.uint64).copy()
    v[np.isnan(a)] = np.uint64(0x7FF8000000000000)
    return v


def rand_doubles(rng: np.random.Generator, n: int, emin: int = -60, emax: int = 60) -> np.ndarray:
    """Random signed doubles with random exponents in [emin, emax] and full
    53-bit mantissas."""
    m = rng.integers(0, 1 << 52, n, dtype=np.int64).astype(np.float64) * 2.0 ** -52 + 1.0
    e = rng.integers(emin, emax + 1, n)
    s = np.where(rng.integers(0, 2, n) == 1, -1.0, 1.0)
    return s * np.ldexp(m, e)


def rand_tails(rng: np.random.Generator, heads: np.ndarray, kmin: int = 0, kmax: int = 60) -> np.ndarray:
    """Tails |x1| ~ |x0| 2^-k, k uniform in [kmin, kmax], random sign and
    mantissa: covers the epsilon-order regimes A..C of the Multiply section."""
    k = rng.integers(kmin, kmax + 1, heads.size)
    m = rng.random(heads.size) + 0.5
    s = np.where(rng.integers(0, 2, heads.size) == 1, -1.0, 1.0)
    return s * np.abs(heads) * m * np.ldexp(1.0, -k)


def isqrt_frac(q: Fraction, bits_: int = 300) -> Fraction:
    """sqrt(q) to within 2^-bits_ relative (floor of a scaled integer sqrt)."""
    if q <= 0:
        return Fraction(0)
    s = 2 * bits_
    num = q.numerator << s
    v = math.isqrt(num // q.denominator)
    return Fraction(v, 1 << bits_)


def fma(a: float, b: float, c: float) -> float:
    """Correctly rounded a*b + c from exact rationals (finite inputs); an
    exact zero is +0 unless both a*b and c are -0 (IEEE 754, round to nearest)."""
    q = F(a) * F(b) + F(c)
    if q == 0:
        prod_neg = (math.copysign(1.0, a) * math.copysign(1.0, b)) < 0
        if prod_neg and math.copysign(1.0, c) < 0 and (a == 0 or b == 0) and c == 0:
            return -0.0
        return 0.0
    return rn(q)


# ------------------------------------------------------------------ binary32

U32 = Fraction(1, 2 ** 24)        # unit roundoff of binary32


def rn32(q: Fraction) -> float:
    """Round a rational to the nearest binary32 value (ties to even), as a
    Python float holding that value; overflow gives +-inf."""
    if q == 0:
        return 0.0
    s = -1.0 if q < 0 else 1.0
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    q_exp = max(e, -126) - 23                       # exponent of the ulp
    m = round(a / Fraction(2) ** q_exp)             # round half to even
    v = float(Fraction(m) * Fraction(2) ** q_exp)
    if v > 3.4028234663852886e38:
        return s * math.inf
    return s * v


def f32(x: float) -> float:
    return float(np.float32(x))


def ulp32(x: float) -> float:
    if x == 0 or not math.isfinite(x):
        return 2.0 ** -149 if x == 0 else math.nan
    m, e = math.frexp(abs(x))
    return 2.0 ** (max(e - 1, -126) - 23)


def split32(v: float):
    """A double as a binary32 twofold: (float(v), float(v - float(v)))."""
    h = f32(v)
    return h, f32(v - h)
