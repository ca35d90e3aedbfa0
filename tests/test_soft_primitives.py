"""The CUDA library's integer binary64 primitives (division, square root,
Two-Sum tail), compiled for the host from the same header, give the same bits
as the CPU's IEEE operations (and the literal Two-Sum sequence) on millions
of random and adversarial cases, also with seeds perturbed to the edge of
their error bound.  CPU only: the GPU parity tests cover the device build."""
import ctypes
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    so = tmp_path_factory.mktemp("soft") / "libsofthost.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared", os.path.join(HERE, "soft_host.cpp"), "-o", str(so)])
    L = ctypes.CDLL(str(so))
    d, i64, u64, p = ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
    for name in ("check_div", "check_sqrt", "check_sum_err", "check_diff_err", "check_twice", "check_mul",
                 "check_add", "check_two_prod", "check_remainders"):
        getattr(L, name).argtypes = [u64, i64, ctypes.c_int, ctypes.c_int, p]
        getattr(L, name).restype = i64
    for name in ("check_div_hard", "check_sqrt_hard", "check_div_by_root", "check_div_shared",
                 "check_sqrt_near", "check_scale_pow2", "check_remainder_specials", "check_div_by_near_root",
                 "check_diff_err_near", "check_two_sum_fp"):
        getattr(L, name).argtypes = [u64, i64, p]
        getattr(L, name).restype = i64
    L.soft_div.argtypes = [d, d]
    L.soft_div.restype = d
    L.soft_sqrt.argtypes = [d]
    L.soft_sqrt.restype = d
    L.soft_sum_err.argtypes = [d, d]
    L.soft_sum_err.restype = d
    L.set_seed_scale.argtypes = [ctypes.c_float]
    return L


def run(H, fn, *args):
    bad = (ctypes.c_double * 2)()
    n = getattr(H, fn)(*args, bad)
    assert n == 0, f"{fn}{args}: {n} mismatches, first {bad[0]!r}, {bad[1]!r}"


SCALES = [1.0, 1.0 + 2 ** -22, 1.0 - 2 ** -22]


@pytest.mark.parametrize("scale", SCALES)
def test_div_matches_ieee(H, scale):
    H.set_seed_scale(scale)
    try:
        run(H, "check_div", 1, 2_000_000, 1000, 1046)      # ordinary exponents
        run(H, "check_div", 2, 1_000_000, 0, 2047)         # everything, incl. specials
        run(H, "check_div", 3, 1_000_000, 1, 60)           # underflowing quotients
        run(H, "check_div", 4, 1_000_000, 1990, 2046)      # overflowing quotients
        run(H, "check_div_hard", 5, 2_000_000)
    finally:
        H.set_seed_scale(1.0)


@pytest.mark.parametrize("scale", SCALES)
def test_sqrt_matches_ieee(H, scale):
    H.set_seed_scale(scale)
    try:
        run(H, "check_sqrt", 6, 2_000_000, 1, 2046)
        run(H, "check_sqrt", 7, 500_000, 0, 2047)
        run(H, "check_sqrt_hard", 8, 2_000_000)
    finally:
        H.set_seed_scale(1.0)


def test_sum_err_matches_literal_two_sum(H):
    run(H, "check_sum_err", 9, 3_000_000, 900, 1150)
    run(H, "check_sum_err", 10, 1_000_000, 0, 2047)
    run(H, "check_sum_err", 11, 1_000_000, 0, 80)        # subnormal and tiny
    run(H, "check_sum_err", 12, 1_000_000, 1980, 2046)   # near overflow


def test_diff_err_matches_literal_two_diff(H):
    run(H, "check_diff_err", 13, 2_000_000, 900, 1150)
    run(H, "check_diff_err", 14, 1_000_000, 0, 2047)
    run(H, "check_diff_err", 15, 1_000_000, 1980, 2046)


def test_fast_two_sum_form_matches_literal_two_sum(H):
    """RTF1's Two-Sum of x0 and x1 as Fast-Two-Sum on exponent-ordered
    operands (device two_sum_fp), restated on the host."""
    run(H, "check_two_sum_fp", 33, 3_000_000)


def test_sterbenz_diff_tail_matches_literal_two_diff(H):
    """RTF1's Two-Diff tail with the exact-difference short cut."""
    run(H, "check_diff_err_near", 32, 2_000_000)


@pytest.mark.parametrize("scale", SCALES)
def test_div_with_reused_reciprocals(H, scale):
    H.set_seed_scale(scale)
    try:
        run(H, "check_div_by_root", 19, 2_000_000)
        run(H, "check_div_shared", 20, 2_000_000)
        run(H, "check_sqrt_near", 29, 2_000_000)
        run(H, "check_div_by_near_root", 31, 2_000_000)
    finally:
        H.set_seed_scale(1.0)


def test_mul_matches_ieee(H):
    run(H, "check_mul", 21, 2_000_000, 900, 1150)
    run(H, "check_mul", 22, 1_000_000, 0, 2047)
    run(H, "check_mul", 23, 500_000, 400, 640)       # products near the underflow threshold
    run(H, "check_mul", 24, 500_000, 1500, 1550)     # products near the overflow threshold


def test_two_prod_matches_mul_and_fma(H):
    run(H, "check_two_prod", 31, 2_000_000, 900, 1150)
    run(H, "check_two_prod", 32, 1_000_000, 0, 2047)
    run(H, "check_two_prod", 33, 500_000, 500, 620)      # errors near the subnormal range
    run(H, "check_two_prod", 34, 500_000, 1500, 1550)    # products near overflow


def test_packed_remainders_match_fma(H):
    run(H, "check_remainders", 35, 2_000_000, 900, 1150)
    run(H, "check_remainders", 36, 1_000_000, 0, 2047)
    run(H, "check_remainders", 37, 500_000, 1, 120)      # remainders near the subnormal range
    run(H, "check_remainder_specials", 0, 0)             # zeros, Inf, NaN, subnormals, extremes


def test_add_matches_ieee(H):
    run(H, "check_add", 25, 3_000_000, 900, 1150)
    run(H, "check_add", 26, 1_000_000, 0, 2047)
    run(H, "check_add", 27, 500_000, 0, 60)          # subnormal and tiny
    run(H, "check_add", 28, 500_000, 2000, 2046)     # near overflow


def test_pow2_scaling_of_thresholds(H):
    run(H, "check_scale_pow2", 30, 2_000_000)


def test_twice_matches_ieee(H):
    run(H, "check_twice", 16, 1_000_000, 0, 2047)
    run(H, "check_twice", 17, 200_000, 0, 2)
    run(H, "check_twice", 18, 200_000, 2044, 2047)


def test_corner_values(H):
    import math
    big = 1.7976931348623157e308
    cases = [(big, -3 * 2.0 ** 970), (-big, 3 * 2.0 ** 970), (3 * 2.0 ** 970, -big), (big, big),
             (5.0, -0.0), (-0.0, -0.0), (0.0, -0.0), (2.0 ** -1074, -(2.0 ** -1074)), (1.0, 2.0 ** -60),
             (1e308, 1e308), (math.inf, 1.0), (math.nan, 1.0), (-math.inf, math.inf)]
    for a, b in cases:
        s = a + b
        bv = s - a
        av = s - bv
        t = (a - av) + (b - bv)
        got = H.soft_sum_err(a, b)
        assert (math.isnan(t) and math.isnan(got)) or (t == got and math.copysign(1, t) == math.copysign(1, got)), (a, b, t, got)
    for a, b in [(1.0, 3.0), (-1.0, 3.0), (2.0 ** 1023, 0.5), (1.0, 2.0 ** 1023), (7.0, 2.0),
                 (2.0 ** -1022, 2.0), (1.0, 0.0), (0.0, 0.0), (math.inf, 2.0), (1.0, math.nan)]:
        ref = a / b if b != 0 else (math.copysign(math.inf, a * b) if a != 0 else math.nan)
        got = H.soft_div(a, b)
        assert (math.isnan(ref) and math.isnan(got)) or ref == got, (a, b, ref, got)
    for a in [4.0, 2.0, 0.25, 2.0 ** -1022, 2.0 ** 1023, 1.7976931348623157e308, 0.0, -0.0, 1.0]:
        assert H.soft_sqrt(a) == math.sqrt(a)
