// Host build of the library's integer binary64 primitives (tf_soft.cuh),
// checked in bulk against the CPU's own IEEE operations and against the
// literal Two-Sum sequence.  Test infrastructure: compiled by
// tests/test_soft_primitives.py with g++ -ffp-contract=off.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "../paper_1401_6235_gb300/csrc/tf_soft.cuh"

using namespace tf::soft;

namespace {

uint64_t mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// random double: exponent field uniform in [elo, ehi], random sign/fraction
double rnd(uint64_t key, uint64_t i, int elo, int ehi) {
    uint64_t r = mix(key + (i + 1) * 0x9E3779B97F4A7C15ULL);
    uint64_t r2 = mix(r ^ 0xD1B54A32D192ED03ULL);
    int e = elo + (int)(r2 % (uint64_t)(ehi - elo + 1));
    uint64_t f = r & kFrac;
    // bias towards edge significands now and then
    switch ((r2 >> 20) & 15) {
    case 0: f = 0; break;
    case 1: f = kFrac; break;
    case 2: f &= 0xFFFF000000000000ull >> 12; break;
    case 3: f |= 0x000FFFFFFF000000ull; break;
    default: break;
    }
    return u2d(((r2 >> 63) << 63) | ((uint64_t)e << 52) | f);
}

bool same(double x, double y) {
    if (std::isnan(x) || std::isnan(y)) return std::isnan(x) && std::isnan(y);
    return d2u(x) == d2u(y);
}

double literal_two_sum_tail(double a, double b) {
    volatile double s = a + b;
    volatile double bv = s - a;
    volatile double av = s - bv;
    volatile double br = b - bv;
    volatile double ar = a - av;
    volatile double t = ar + br;
    return t;
}

double literal_two_diff_tail(double a, double b) {
    volatile double d = a - b;
    volatile double bv = a - d;
    volatile double av = bv + d;
    volatile double br = bv - b;
    volatile double ar = a - av;
    volatile double t = ar + br;
    return t;
}

}  // namespace

extern "C" {

void set_seed_scale(float s) { host_seed_scale() = s; }

double soft_div(double a, double b) { return div_rn(a, b); }
double soft_sqrt(double a) { return sqrt_rn(a); }
double soft_sum_err(double a, double b) { return sum_err(a, b, native_add(a, b)); }

int64_t check_twice(uint64_t key, int64_t n, int elo, int ehi, double *bad) {
    int64_t nbad = 0;
    for (int64_t i = 0; i < n; ++i) {
        double c = rnd(key, i, elo, ehi);
        volatile double ref = 2.0 * c;
        if (!same(twice(c), ref)) {
            if (!nbad) bad[0] = c;
            ++nbad;
        }
    }
    return nbad;
}

// Mismatch counts over n random cases; the first bad pair goes to bad[0..1].
int64_t check_div(uint64_t key, int64_t n, int elo, int ehi, double *bad) {
    int64_t nbad = 0;
    for (int64_t i = 0; i < n; ++i) {
        double a = rnd(key, 2 * i, elo, ehi), b = rnd(key, 2 * i + 1, elo, ehi);
        volatile double ref = a / b;
        if (!same(div_rn(a, b), ref)) {
            if (!nbad) { bad[0] = a; bad[1] = b; }
            ++nbad;
        }
    }
    return nbad;
}

int64_t check_sqrt(uint64_t key, int64_t n, int elo, int ehi, double *bad) {
    int64_t nbad = 0;
    for (int64_t i = 0; i < n; ++i) {
        double a = std::fabs(rnd(key, i, elo, ehi));
        volatile double ref = std::sqrt(a);
        if (!same(sqrt_rn(a), ref)) {
            if (!nbad) bad[0] = a;
            ++nbad;
        }
    }
    return nbad;
}

// Two-Sum tail: exponents of a and b drawn independently in [elo, ehi]
// (gaps of any size), compared with the literal six-operation sequence.
int64_t check_sum_err(uint64_t key, int64_t n, int elo, int ehi, double *bad) {
    int64_t nbad = 0;
    for (int64_t i = 0; i < n; ++i) {
        double a = rnd(key, 2 * i, elo, ehi), b = rnd(key, 2 * i + 1, elo, ehi);
        if (i & 1) b = -a * (1.0 + std::ldexp((double)(i % 97), -50));   // heavy cancellation
        if (i % 5 == 0) b = std::ldexp(a, -(int)(i % 70));                 // controlled gaps
        double ref = literal_two_sum_tail(a, b);
        double got = sum_err(a, b, native_add(a, b));
        if (!same(got, ref)) {
            if (!nbad) { bad[0] = a; bad[1] = b; }
            ++nbad;
        }
    }
    return nbad;
}

// Two-Diff tail (Shewchuk's order) equals the Two-Sum tail of (a, -b, a - b).
int64_t check_diff_err(uint64_t key, int64_t n, int elo, int ehi, double *bad) {
    int64_t nbad = 0;
    for (int64_t i = 0; i < n; ++i) {
        double a = rnd(key, 2 * i, elo, ehi), b = rnd(key, 2 * i + 1, elo, ehi);
        if (i & 1) b = a * (1.0 + std::ldexp((double)(i % 97), -50));
        if (i % 5 == 0) b = std::ldexp(a, -(int)(i % 70));
        volatile double d = a - b;
        double ref = literal_two_diff_tail(a, b);
        double got = sum_err(a, -b, d);
        if (!same(got, ref)) {
            if (!nbad) { bad[0] = a; bad[1] = b; }
            ++nbad;
        }
    }
    return nbad;
}

// Quotients near rounding boundaries: b random, q a random double, a the
// product q*b rounded, nudged by a few ulps.
int64_t check_div_hard(uint64_t key, int64_t n, double *bad) {
    int64_t nbad = 0;
    for (int64_t i = 0; i < n; ++i) {
        double b = rnd(key, 2 * i, 1000, 1046), q = rnd(key, 2 * i + 1, 1000, 1046);
        double a = q * b;
        uint64_t ua = d2u(a) + (int64_t)(i % 7) - 3;
        a = u2d(ua);
        volatile double ref = a / b;
        if (!same(div_rn(a, b), ref)) {
            if (!nbad) { bad[0] = a; bad[1] = b; }
            ++nbad;
        }
    }
    return nbad;
}

// Division by 2 sqrt(u) with the reciprocal square root that sqrt_rn_y
// returns (as in RPF1), against the CPU's t / (2 sqrt(u)).
int64_t check_div_by_root(uint64_t key, int64_t n, double *bad) {
    int64_t nbad = 0;
    for (int64_t i = 0; i < n; ++i) {
        double u = std::fabs(rnd(key, 2 * i, 1, 2046));
        double t = rnd(key, 2 * i + 1, 1, 2046);
        if (i % 3 == 0) t = std::ldexp(t, -(int)(i % 60));
        uint64_t y;
        double c = sqrt_rn_y(u, &y);
        double got = div_rn_y(t, twice(c), y);
        volatile double c2 = std::sqrt(u);
        volatile double w = 2.0 * c2;
        volatile double ref = t / w;
        if (!same(got, ref)) {
            if (!nbad) { bad[0] = t; bad[1] = u; }
            ++nbad;
        }
    }
    return nbad;
}

// Two divisions sharing the divisor's reciprocal (as in DTF1).
int64_t check_div_shared(uint64_t key, int64_t n, double *bad) {
    int64_t nbad = 0;
    for (int64_t i = 0; i < n; ++i) {
        double a = rnd(key, 3 * i, 900, 1150), c = rnd(key, 3 * i + 1, 800, 1150);
        double b = rnd(key, 3 * i + 2, 900, 1150);
        uint64_t y = recip_of(b);
        volatile double r1 = a / b, r2 = c / b;
        if (!same(div_rn_y(a, b, y), r1) || !same(div_rn_y(c, b, y), r2)) {
            if (!nbad) { bad[0] = a; bad[1] = b; }
            ++nbad;
        }
    }
    return nbad;
}

int64_t check_mul(uint64_t key, int64_t n, int elo, int ehi, double *bad) {
    int64_t nbad = 0;
    for (int64_t i = 0; i < n; ++i) {
        double a = rnd(key, 2 * i, elo, ehi), b = rnd(key, 2 * i + 1, elo, ehi);
        if (i % 11 == 5 && elo > 300 && ehi < 1700) {   // ties to even (see check_two_prod)
            a = u2d(0x3FF0000000000001ull + 2 * (mix(key + i) % (1ull << 50)));
            b = std::ldexp(1.5, (int)(i % 60) - 30);
        }
        volatile double ref = a * b;
        if (!same(mul_rn(a, b), ref)) {
            if (!nbad) { bad[0] = a; bad[1] = b; }
            ++nbad;
        }
    }
    return nbad;
}

int64_t check_add(uint64_t key, int64_t n, int elo, int ehi, double *bad) {
    int64_t nbad = 0;
    for (int64_t i = 0; i < n; ++i) {
        double a = rnd(key, 2 * i, elo, ehi), b = rnd(key, 2 * i + 1, elo, ehi);
        if (i % 3 == 1) b = -a * (1.0 + std::ldexp((double)(i % 97), -52));   // cancellation
        if (i % 5 == 0) b = std::ldexp(a, -(int)(i % 70));                     // controlled gaps
        if (i % 7 == 0) b = -std::ldexp(a, -(int)(i % 66));
        volatile double ref = a + b;
        if (!same(add_rn(a, b), ref)) {
            if (!nbad) { bad[0] = a; bad[1] = b; }
            ++nbad;
        }
    }
    return nbad;
}

// sqrt(u) from the reciprocal root of sqrt(x) for u within a few hundred
// ulps of x (RTF1's second root), including binade crossings and far
// values that take the full path.
int64_t check_sqrt_near(uint64_t key, int64_t n, double *bad) {
    int64_t nbad = 0;
    for (int64_t i = 0; i < n; ++i) {
        double x = std::fabs(rnd(key, i, 1, 2046));
        int64_t k = (int64_t)(mix(key ^ (uint64_t)i) % 1200) - 600;   // ulps, some beyond 256
        if (i % 11 == 0) x = u2d((d2u(x) & ~kFrac) | (i & 1 ? 0 : kFrac));   // binade edges
        double u = u2d(d2u(x) + k);
        if (!(u > 0) || std::isinf(u)) continue;
        uint64_t yx;
        (void)sqrt_rn_y(x, &yx);
        volatile double ref = std::sqrt(u);
        if (!same(sqrt_rn_near(u, x, yx), ref)) {
            if (!nbad) { bad[0] = u; bad[1] = x; }
            ++nbad;
        }
    }
    return nbad;
}

// RN(|z| 2^k) from bits against the CPU's ldexp-free multiplication.
int64_t check_scale_pow2(uint64_t key, int64_t n, double *bad) {
    int64_t nbad = 0;
    for (int64_t i = 0; i < n; ++i) {
        double z = rnd(key, i, 0, 2047);
        int k = -(int)(mix(key + i) % 1100);
        volatile double t = std::ldexp(1.0, k < -1022 ? -1022 : k);
        if (k < -1022) continue;
        volatile double ref = std::fabs(z) * t;
        uint64_t got = scale_abs_pow2(d2u(z), k);
        if (!same(u2d(got), ref)) {
            if (!nbad) { bad[0] = z; bad[1] = (double)k; }
            ++nbad;
        }
    }
    return nbad;
}

// Two-Product pair against the CPU's multiplication and fma(a, b, -p).
int64_t check_two_prod(uint64_t key, int64_t n, int elo, int ehi, double *bad) {
    int64_t nbad = 0;
    for (int64_t i = 0; i < n; ++i) {
        double a = rnd(key, 2 * i, elo, ehi), b = rnd(key, 2 * i + 1, elo, ehi);
        if (i % 9 == 0) b = std::ldexp(1.0, (int)(i % 40) - 20);        // exact products
        if (i % 13 == 0) a = 0.0;
        if (i % 11 == 5) {   // ties: an odd significand below 4/3 times 1.5: the low half is exactly 2^51
            a = u2d(0x3FF0000000000001ull + 2 * (mix(key + i) % (1ull << 50)));
            b = std::ldexp(1.5, (int)(i % 60) - 30) * (i & 1 ? -1.0 : 1.0);
        }
        volatile double pr = a * b;
        volatile double er = std::fma(a, b, -pr);
        double p, e;
        two_prod_rn(a, b, p, e);
        if (!same(p, pr) || !same(e, er)) {
            if (!nbad) { bad[0] = a; bad[1] = b; }
            ++nbad;
        }
    }
    return nbad;
}

// Remainders packed from the integer division / root against fma.
int64_t check_remainders(uint64_t key, int64_t n, int elo, int ehi, double *bad) {
    int64_t nbad = 0;
    for (int64_t i = 0; i < n; ++i) {
        double a = rnd(key, 2 * i, elo, ehi), b = rnd(key, 2 * i + 1, elo, ehi);
        double r;
        double q = div_rn_y(a, b, 0, &r);
        volatile double qr = a / b;
        volatile double rr = std::fma(-qr, b, a);
        double x = std::fabs(a);
        uint64_t y;
        double dx;
        const double cx = sqrt_rn_y(x, &y, &dx);
        volatile double cxr = std::sqrt(x);
        volatile double dxr = std::fma(-cxr, cxr, x);
        if (!same(cx, cxr) || !same(dx, dxr)) {
            if (!nbad) { bad[0] = x; bad[1] = 0.0; }
            ++nbad;
        }
        double u = u2d(d2u(x) + (int64_t)(i % 401) - 200);
        double d;
        double v = sqrt_rn_near(u, x, y, &d);
        volatile double vr = std::sqrt(u);
        volatile double dr = std::fma(-vr, vr, u);
        if (!same(q, qr) || !same(r, rr) || !same(v, vr) || !same(d, dr)) {
            if (!nbad) { bad[0] = a; bad[1] = b; }
            ++nbad;
        }
    }
    return nbad;
}

// Perfect squares and their neighbours.
int64_t check_sqrt_hard(uint64_t key, int64_t n, double *bad) {
    int64_t nbad = 0;
    for (int64_t i = 0; i < n; ++i) {
        double r = std::fabs(rnd(key, i, 500, 1500));
        double a = r * r;
        if (!(a > 0) || std::isinf(a)) continue;
        uint64_t ua = d2u(a) + (int64_t)(i % 5) - 2;
        a = u2d(ua);
        volatile double ref = std::sqrt(a);
        if (!same(sqrt_rn(a), ref)) {
            if (!nbad) bad[0] = a;
            ++nbad;
        }
    }
    return nbad;
}

// Remainders of the special cases (zeros, Inf, NaN, subnormals, extremes):
// every ordered pair of a fixed list, for the division and for the root of
// u started from x's reciprocal root (sqrt_rn_near falls back on its own).
int64_t check_remainder_specials(uint64_t key, int64_t n, double *bad) {
    (void)key;
    (void)n;
    const double inf = INFINITY, big = 1.7976931348623157e308, tiny = 4.9406564584124654e-324;
    const double vals[] = {0.0, -0.0, inf, -inf, NAN, -NAN, 1.0, -1.0, 3.0, -0.75, big, -big, tiny, -tiny,
                           2.2250738585072014e-308, 1e-310, -3e-320, 2.0, 0.5, 1e300, -1e-300};
    const int nv = (int)(sizeof(vals) / sizeof(vals[0]));
    int64_t nbad = 0;
    for (int i = 0; i < nv; ++i) {
        for (int j = 0; j < nv; ++j) {
            const double a = vals[i], b = vals[j];
            double r;
            const double q = div_rn_y(a, b, 0, &r);
            volatile double qr = a / b;
            volatile double rr = std::fma(-qr, b, a);
            uint64_t y;
            (void)sqrt_rn_y(b, &y);
            double d;
            const double v = sqrt_rn_near(a, b, y, &d);
            volatile double vr = std::sqrt(a);
            volatile double dr = std::fma(-vr, vr, a);
            uint64_t ya;
            double da;
            const double va = sqrt_rn_y(a, &ya, &da);
            if (!same(q, qr) || !same(r, rr) || !same(v, vr) || !same(d, dr) || !same(va, vr) || !same(da, dr)) {
                if (!nbad) { bad[0] = a; bad[1] = b; }
                ++nbad;
            }
        }
    }
    return nbad;
}

// RPF1's division by 2 v inside RTF1: v = sqrt(u) for u within a few hundred
// ulps of x (binade edges included, some far enough for the full root),
// divided with the reciprocal estimate sqrt_rn_near hands out, against the
// CPU's t / (2 sqrt(u)).
int64_t check_div_by_near_root(uint64_t key, int64_t n, double *bad) {
    int64_t nbad = 0;
    for (int64_t i = 0; i < n; ++i) {
        double x = std::fabs(rnd(key, 2 * i, 1, 2046));
        int64_t k = (int64_t)(mix(key ^ (uint64_t)i) % 1200) - 600;
        if (i % 11 == 0) x = u2d((d2u(x) & ~kFrac) | (i & 1 ? 0 : kFrac));
        double u = u2d(d2u(x) + k);
        if (!(u > 0) || std::isinf(u)) continue;
        double t = rnd(key, 2 * i + 1, 1, 2046);
        if (i % 3 == 0) t = std::ldexp(t, -(int)(i % 60));
        uint64_t yx, yv;
        (void)sqrt_rn_y(x, &yx);
        double d;
        const double v = sqrt_rn_near(u, x, yx, &d, &yv);
        const double got = div_rn_y(t, twice(v), yv);
        volatile double vr = std::sqrt(u);
        volatile double w = 2.0 * vr;
        volatile double ref = t / w;
        if (!same(v, vr) || !same(got, ref)) {
            if (!nbad) { bad[0] = t; bad[1] = u; }
            ++nbad;
        }
    }
    return nbad;
}

// The Two-Diff tail with the Sterbenz short cut against the literal
// sequence: pairs in one binade (the short cut), neighbours across a binade
// edge, random pairs, and a fixed list of special values (zeros of both
// signs, subnormals, Inf, NaN, the largest finite values).
int64_t check_diff_err_near(uint64_t key, int64_t n, double *bad) {
    int64_t nbad = 0;
    const double inf = INFINITY, big = 1.7976931348623157e308;
    const double vals[] = {0.0, -0.0, inf, -inf, NAN, 1.0, -1.0, 1.5, big, -big, 4.9406564584124654e-324,
                           -1e-310, 1e-310, 2.2250738585072014e-308, 2.0, 0.75};
    const int nv = (int)(sizeof(vals) / sizeof(vals[0]));
    for (int64_t i = 0; i < n + nv * nv; ++i) {
        double a, b;
        if (i >= n) {
            a = vals[(i - n) / nv];
            b = vals[(i - n) % nv];
        } else {
            a = rnd(key, 2 * i, 1, 2046);
            if (i % 3 == 0) b = u2d(d2u(a) + (int64_t)(mix(key + i) % 2000) - 1000);      // one binade, mostly
            else if (i % 3 == 1) b = u2d((d2u(a) & ~kFrac) - (i & 2 ? 1 : 0));             // a binade edge
            else b = rnd(key, 2 * i + 1, 1, 2046);
        }
        volatile double d = a - b;
        const double ref = literal_two_diff_tail(a, b);
        const double got = u2d(diff_err_near_bits(d2u(a), d2u(b), d2u(d)));
        if (!same(got, ref)) {
            if (!nbad) { bad[0] = a; bad[1] = b; }
            ++nbad;
        }
    }
    return nbad;
}

// The device's Fast-Two-Sum form of the Two-Sum tail (two_sum_fp in
// tf_device.cuh: operands ordered by exponent field, small - (s - big), a
// zero made +0; fields >= 2045 take sum_err) restated with host doubles,
// against the literal Two-Sum sequence: random pairs over the whole range,
// pairs with small gaps, cancellations, subnormals and special values.
int64_t check_two_sum_fp(uint64_t key, int64_t n, double *bad) {
    int64_t nbad = 0;
    const double vals[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, 1.0, -1.0, 1.7976931348623157e308,
                           -1.7976931348623157e308, 4.9406564584124654e-324, -1e-310, 2.2250738585072014e-308};
    const int nv = (int)(sizeof(vals) / sizeof(vals[0]));
    for (int64_t i = 0; i < n + nv * nv; ++i) {
        double a, b;
        if (i >= n) {
            a = vals[(i - n) / nv];
            b = vals[(i - n) % nv];
        } else {
            a = rnd(key, 2 * i, 0, 2047);
            b = rnd(key, 2 * i + 1, 0, 2047);
            if (i % 3 == 1) b = -a * (1.0 + std::ldexp((double)(i % 97), -52));
            if (i % 5 == 0) b = std::ldexp(a, -(int)(i % 70)) * (i & 8 ? -1.0 : 1.0);
        }
        volatile double s = a + b;
        const double ref = literal_two_sum_tail(a, b);
        const uint64_t ua = d2u(a), ub = d2u(b);
        const unsigned fa = (unsigned)(ua >> 52) & 0x7FF, fb = (unsigned)(ub >> 52) & 0x7FF;
        double got;
        if ((fa >= 2045) | (fb >= 2045)) {
            got = sum_err(a, b, s);
        } else {
            const bool sw = fb > fa;
            const double big = sw ? b : a, small = sw ? a : b;
            volatile double z = s - big;
            volatile double tt = small - z;
            const uint64_t ut = d2u(tt);
            got = u2d((ut << 1) ? ut : 0);
        }
        if (!same(got, ref)) {
            if (!nbad) { bad[0] = a; bad[1] = b; }
            ++nbad;
        }
    }
    return nbad;
}

}  // extern "C"
