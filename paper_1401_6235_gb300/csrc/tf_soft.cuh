// Correctly rounded binary64 primitives computed on the integer pipes.
//
// On GB300 the FP64 pipe issues about 2 operations per clock per SM while
// the integer pipes issue about 90; a native __ddiv_rn or __dsqrt_rn costs
// about 8.5 FP64 issue slots.  The functions below produce the SAME bits as
// the native round-to-nearest-even operation (IEEE 754 binary64) but do the
// work with 32/64-bit integer instructions and one single-precision seed from
// the special-function unit:
//
//   div_rn(a, b)        a / b
//   sqrt_rn(a)          sqrt(a)
//   sum_err(a, b, s)    a + b - s exactly, for s = RN(a + b)   (Two-Sum tail)
//
// Each has a fast path for the ordinary case (normal operands and result)
// and falls back to the native instruction otherwise (zeros, subnormals,
// Inf, NaN, results near the overflow or underflow thresholds), so the
// result is always the IEEE result.  Division and square root use the
// classic scheme: a reciprocal (square-root reciprocal) seed, two
// Newton-Raphson steps in 64-bit fixed point, a quotient (root) estimate
// within one unit, and an exact integer remainder that corrects the
// estimate and decides the rounding (Markstein-style correction; see e.g.
// Muller et al., Handbook of Floating-Point Arithmetic, ch. 9 and 10).
//
// The header also compiles as plain C++ (no CUDA) so the host test suite can
// check the integer algorithms against the CPU's IEEE operations; there the
// seeds come from correctly rounded float operations.
#pragma once
#if !defined(__CUDACC_RTC__)   // the runtime compiler gets the integer types from its prelude
#include <cstdint>
#include <cstring>
#include <cmath>
#endif

#if defined(__CUDACC__)
#define TFS_HD __host__ __device__ __forceinline__
#define TFS_COLD static __host__ __device__ __noinline__   // rare paths: kept out of the hot code
#else
#define TFS_HD inline
#define TFS_COLD static inline
#endif

namespace tf {
namespace soft {

constexpr uint64_t kFrac = 0x000FFFFFFFFFFFFFull;
constexpr uint64_t kHid = 0x0010000000000000ull;
constexpr uint64_t kSign = 0x8000000000000000ull;

// Bit moves between binary64 and integer registers.  On the device they are
// opaque register moves (inline PTX), so that the compiler does not turn a
// sign-bit mask or flip on the bits into a floating-point absolute value or
// negation, which it would issue on the FP64 pipe (one FP64 instruction
// each); with the moves opaque, sign work stays on the integer pipes.
TFS_HD uint64_t d2u(double x) {
#if defined(__CUDA_ARCH__)
    uint64_t u;
    asm("mov.b64 %0, %1;" : "=l"(u) : "d"(x));
    return u;
#else
    uint64_t u;
    std::memcpy(&u, &x, 8);
    return u;
#endif
}

TFS_HD double u2d(uint64_t u) {
#if defined(__CUDA_ARCH__)
    double x;
    asm("mov.b64 %0, %1;" : "=d"(x) : "l"(u));
    return x;
#else
    double x;
    std::memcpy(&x, &u, 8);
    return x;
#endif
}

TFS_HD uint64_t mulhi(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

TFS_HD int clz64(uint64_t v) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

// (x y) >> 64 from the three largest 32 x 32-bit products (the low one
// dropped): at most 1 below the exact value.  Cheaper than the full high
// product where a routine's error budget absorbs the unit.
TFS_HD uint64_t mulhi3(uint64_t x, uint64_t y) {
    const uint64_t x1 = x >> 32, x0 = x & 0xFFFFFFFFull, y1 = y >> 32, y0 = y & 0xFFFFFFFFull;
    const uint64_t m1 = x1 * y0, m2 = x0 * y1;
    return x1 * y1 + (m1 >> 32) + (m2 >> 32) + (((m1 & 0xFFFFFFFFull) + (m2 & 0xFFFFFFFFull)) >> 32);
}

// (x y) >> 64 from the high words alone, below the exact value by less than
// 2^33: for quotient corrections whose scale makes that a fraction of a unit.
TFS_HD uint64_t mulhi1(uint64_t x, uint64_t y) { return (x >> 32) * (y >> 32); }

// Seed tests may perturb on the host: relative factor applied to seeds.
#if !defined(__CUDA_ARCH__)
inline float &host_seed_scale() {
    static float s = 1.0f;
    return s;
}
#endif

// 1/f for f in [2^23, 2^24), relative error below 2^-22.
TFS_HD float rcp_seed(float f) {
#if defined(__CUDA_ARCH__)
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(f));
    return r;
#else
    return (1.0f / f) * host_seed_scale();
#endif
}

// 1/sqrt(f) for f in [2^22, 2^24), relative error below 2^-22.
TFS_HD float rsqrt_seed(float f) {
#if defined(__CUDA_ARCH__)
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(f));
    return r;
#else
    return (1.0f / std::sqrt(f)) * host_seed_scale();
#endif
}

TFS_HD float u2f(uint32_t u) {
#if defined(__CUDA_ARCH__)
    return __uint_as_float(u);
#else
    float f;
    std::memcpy(&f, &u, 4);
    return f;
#endif
}

TFS_HD uint32_t f2u(float f) {
#if defined(__CUDA_ARCH__)
    return __float_as_uint(f);
#else
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
#endif
}

// The native fallbacks are volatile inline PTX on the device, so that the
// compiler never evaluates them speculatively on lanes that do not take the
// fallback branch (a native division or root is ~8 FP64 issue slots).
TFS_HD double native_div(double a, double b) {
#if defined(__CUDA_ARCH__)
    double r;
    asm volatile("div.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b));
    return r;
#else
    volatile double r = a / b;
    return r;
#endif
}

TFS_HD double native_sqrt(double a) {
#if defined(__CUDA_ARCH__)
    double r;
    asm volatile("sqrt.rn.f64 %0, %1;" : "=d"(r) : "d"(a));
    return r;
#else
    volatile double r = std::sqrt(a);
    return r;
#endif
}

TFS_HD double native_add(double a, double b) {
#if defined(__CUDA_ARCH__)
    double r;
    asm volatile("add.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b));
    return r;
#else
    volatile double r = a + b;
    return r;
#endif
}

TFS_HD double native_fma(double a, double b, double c) {
#if defined(__CUDA_ARCH__)
    double r;
    asm volatile("fma.rn.f64 %0, %1, %2, %3;" : "=d"(r) : "d"(a), "d"(b), "d"(c));
    return r;
#else
    volatile double r = std::fma(a, b, c);
    return r;
#endif
}

// A seed y = m * 2^(e-150) (m the 24-bit significand, e the biased
// exponent) for w in (1, 2] as the fixed-point value w 2^63 = m << (e - bias);
// a seed at or above w = 2 (shift 41) saturates to 2^64 - 1.
TFS_HD uint64_t float_fixed(float y, int bias) {
    const uint32_t u = f2u(y);
    const uint64_t m = (uint64_t)((u & 0x7FFFFFu) | 0x800000u);
    const int sh = (int)((u >> 23) & 0xFFu) - bias;
    return sh >= 41 ? ~0ull : (m << sh);
}

// (a 2^32 + b) * m >> k for 0 <= k <= 32, a, b < 2^32, m < 2^24: the high
// bits of a 64 x 24-bit product from two 32 x 32-bit products.  Sets *ovf
// when the result does not fit 64 bits.
TFS_HD uint64_t mul_m24_shr(uint64_t x, uint64_t m, int k, bool *ovf) {
    const uint64_t A = (x >> 32) * m, B = (x & 0xFFFFFFFFull) * m;   // each < 2^56
    const uint64_t hi = A << (32 - k), lo = B >> k;
    *ovf = (A >> (32 + k)) != 0 || hi + lo < hi;
    return hi + lo;
}

// Y ~ 2^116 / mb (1/d in 1.63 fixed point, d = mb / 2^53 in [1/2, 1)) from
// the single-precision seed and ONE Newton step, both products taken with
// the 24-bit seed significand m: Y never exceeds the true value by more
// than 2^-61 relative and is below it by at most 2^-43.  (Newton's step
// from below-by-eps lands below-by-eps^2; eps <= 2^-22 for the seed.)
TFS_HD uint64_t recip1(uint64_t mb) {
    const uint32_t v = (uint32_t)(mb >> 29);                   // [2^23, 2^24)
    const uint32_t ru = f2u(rcp_seed(u2f(0x4B000000u | (v & 0x7FFFFFu))));
    uint64_t m = (uint64_t)((ru & 0x7FFFFFu) | 0x800000u);
    int sh = (int)((ru >> 23) & 0xFFu) - 63;                   // y0 = m << sh, sh = 40 or 41
    if (sh >= 41) { m = 0xFFFFFFull; sh = 40; }                // w at 2: 2^64 - 2^40
    bool ovf;
    const uint64_t t = mul_m24_shr(mb << 11, m, 64 - sh, &ovf);   // d w0 2^63
    const uint64_t e = 0 - t;                                      // (2 - d w0) 2^63
    const uint64_t y = mul_m24_shr(e, m, 63 - sh, &ovf);           // w0 (2 - d w0) 2^63
    return ovf ? ~0ull : y;
}

// The significand of b in [2^52, 2^53) (meaningful for normal b only).
TFS_HD uint64_t signif(double b) { return (d2u(b) & kFrac) | kHid; }

// Reciprocal of b's significand for div_rn_y; any normal b.
TFS_HD uint64_t recip_of(double b) { return recip1(signif(b)); }

// Bits of the exact value v 2^scale for a signed integer |v| < 2^54 with at
// most 53 significant bits; false when the value would not be a normal
// binary64 (the caller then uses the native operation).  v = 0 gives +0.
TFS_HD bool pack_exact(int64_t v, int scale, uint64_t *out) {
    if (v == 0) { *out = 0; return true; }
    const uint64_t sign = v < 0 ? kSign : 0;
    const uint64_t mag = (uint64_t)(v < 0 ? -v : v);
    const int lz = clz64(mag);
    const int lead = 63 - lz + scale;
    if (lead < -1022 || lead > 1023) return false;
    *out = sign | ((uint64_t)(lead + 1023) << 52) | (((mag << lz) >> 11) & kFrac);
    return true;
}

// Correctly rounded a / b given y, an estimate of 2^116 / signif(b) with
// relative error below 2^-52 (recip_of(b), or the reciprocal square root of
// sqrt_rn_y when b is twice that root), or 0 to compute it here: the
// quotient estimate is then within two units and the remainder corrections
// below restore the exact quotient.
// With rem != nullptr, *rem also receives RN(a - q b) for the returned q,
// the bits of fma(-q, b, a) (Algorithm 4's exact remainder).
TFS_HD double div_rn_y(double a, double b, uint64_t y_in, double *rem = nullptr);

// Correctly rounded a / b.
TFS_HD double div_rn(double a, double b) { return div_rn_y(a, b, 0); }

TFS_HD double div_rn_y(double a, double b, uint64_t y_in, double *rem) {
    const uint64_t ua = d2u(a), ub = d2u(b);
    const int ea = (int)((ua >> 52) & 0x7FF), eb = (int)((ub >> 52) & 0x7FF);
    const int ed = ea - eb;
    // ordinary case: normal operands, quotient normal and finite before and
    // after rounding (field of the result = ed + 1023 - sh lies in [1, 2045])
    if ((unsigned)(ea - 1) >= 2046u || (unsigned)(eb - 1) >= 2046u || ed < -1021 || ed > 1022) {
        // IEEE special cases in integer form (no native instruction, so
        // lanes holding NaN or Inf do not make the whole warp run one);
        // subnormal operands and quotients near the range limits go native.
        const uint64_t xa = ua & ~kSign, xb = ub & ~kSign, inf = 0x7FF0000000000000ull;
        const uint64_t sign = (ua ^ ub) & kSign;
        // The remainder fma(-q, b, a) of these cases is NaN (an Inf or NaN
        // operand, or a zero divisor: Inf - Inf or 0 * Inf) except for a zero
        // dividend over a finite nonzero divisor, where -q b and a are zeros
        // of opposite signs and the sum is +0 (a zero over Inf: 0 * Inf).
        const uint64_t nan = 0x7FF8000000000000ull;
        if (xa > inf || xb > inf || (xa == inf && xb == inf) || (xa == 0 && xb == 0)) {
            if (rem) *rem = u2d(nan);
            return u2d(nan);
        }
        if (xa == inf || xb == 0) {
            if (rem) *rem = u2d(nan);
            return u2d(sign | inf);
        }
        if (xa == 0 || xb == inf) {
            if (rem) *rem = u2d(xa == 0 && xb != inf ? 0 : nan);
            return u2d(sign);
        }
        const double q = native_div(a, b);
        if (rem) *rem = native_fma(u2d(d2u(q) ^ kSign), b, a);
        return q;
    }
    const uint64_t ma = (ua & kFrac) | kHid, mb = (ub & kFrac) | kHid;
    const int sh = ma < mb;                              // quotient of significands < 1
    uint64_t y = y_in;
    if (!y) y = recip1(mb);
    // Q = floor(ma 2^(52+sh) / mb) = floor(ma w 2^(sh-1)), estimated from
    // (ma 2^11)(w 2^63)/2^64.  y is at most 2^-52 above 1/d (the reciprocal
    // root of a rounded square root; recip1 is within 2^-61) and at most
    // 2^-43 below, so the estimate is at most 3 units above and 2^10 below
    // Q: q - 4 is below Q and the remainder N - q mb lies in [mb, 2^63.01),
    // exact modulo 2^64.
    // (mulhi3 is at most one unit low before the shift: the estimate stays
    // within those bounds up to one more unit below, and the remainder
    // below 2^63.01)
    uint64_t q = (mulhi3(ma << 11, y) >> (11 - sh)) - 4;
    uint64_t r = (ma << (52 + sh)) - q * mb;
    // one correction step dq ~ r / mb = r y / 2^116, off by at most one (the
    // high-word product is low by under 2^33, 2^-19 units of dq)
    const uint64_t dq = mulhi1(r, y) >> 52;
    q += dq;
    r -= dq * mb;
    if ((int64_t)r < 0) { q -= 1; r += mb; }
    if (r >= mb) { q += 1; r -= mb; }
    // round to nearest, ties to even (2r == mb cannot occur for binary64
    // significands, but the rule is kept complete)
    const uint64_t r2 = r << 1;
    const uint64_t up = (r2 > mb) | ((r2 == mb) & (q & 1));
    q += up;
    const uint64_t sign = (ua ^ ub) & kSign;
    const double quo = u2d(sign | (((uint64_t)(ed + 1022 - sh) << 52) + q));
    if (rem) {
        // a - q b = (N - q mb) 2^(Ea - 104 - sh), sign of a; N - q mb = r, or r - mb after rounding up
        const int64_t rs = up ? (int64_t)r - (int64_t)mb : (int64_t)r;
        uint64_t rb;
        if (pack_exact(rs, ea - 1023 - 104 - sh, &rb)) *rem = u2d(rb ^ (rs != 0 ? (ua & kSign) : 0));
        else *rem = native_fma(u2d(d2u(quo) ^ kSign), b, a);
    }
    return quo;
}

// Correctly rounded sqrt(a); *y_out receives 1/sqrt(m) as w 2^63 (m the
// normalised radicand significand), which estimates 2^116 / signif(sqrt(a))
// within 2^-52 relative (0 when the special-value path was taken).
// With rem != nullptr, *rem also receives RN(a - c^2) for the returned root
// c, the bits of fma(-c, c, a) (Algorithm 5's exact residual).
TFS_HD double sqrt_rn_y(double a, uint64_t *y_out, double *rem = nullptr);

TFS_HD double sqrt_rn(double a) {
    uint64_t y;
    return sqrt_rn_y(a, &y);
}

TFS_HD double sqrt_rn_y(double a, uint64_t *y_out, double *rem) {
    *y_out = 0;
    const uint64_t u = d2u(a);
    const int f = (int)(u >> 52);                        // sign and exponent field
    if ((unsigned)(f - 1) >= 2046u) {
        // IEEE special cases in integer form; positive subnormals go native.
        // Residuals: a for a zero (-0 * 0 + 0 keeps the zero's sign), NaN
        // for a negative radicand, Inf (-Inf + Inf) or NaN.
        if ((u << 1) == 0) {                                   // sqrt(+-0) = +-0
            if (rem) *rem = a;
            return a;
        }
        if ((u >> 63) || f == 0x7FF) {
            if (rem) *rem = u2d(0x7FF8000000000000ull);
            return (u >> 63) ? u2d(0x7FF8000000000000ull) : a;   // negative or -NaN; +Inf, +NaN
        }
        const double c = native_sqrt(a);
        if (rem) *rem = native_fma(u2d(d2u(c) ^ kSign), c, a);
        return c;
    }
    const uint64_t mx = (u & kFrac) | kHid;
    const int odd = f & 1;                               // unbiased exponent even
    const int s = odd ? 52 : 53;
    // M = mx 2^s in [2^104, 2^106); Q = floor(sqrt(M)) in [2^52, 2^53)
    const uint64_t m_hi = mx >> (64 - s), m_lo = mx << s;
    const uint64_t mt = (m_hi << 22) | (m_lo >> 42);     // m 2^64, m = M / 2^106 in [1/4, 1)
    // w = 1/sqrt(m) in (1, 2] as Y = w 2^63; seed rsqrt(mt / 2^40) = w 2^-12
    uint64_t y = float_fixed(rsqrt_seed((float)(uint32_t)(mt >> 40)), 75);
    // Newton steps w' = w (3 - m w^2)/2 (never above 1/sqrt(m)).  The first
    // starts from the 24-bit seed and runs on high words only (each product
    // low by under 2^-29 relative), which leaves w within ~2^-28; the second
    // takes three-word products (low by at most one unit) and lands within
    // ~2^-56 below 1/sqrt(m).
    {
        const uint64_t w2 = mulhi1(y, y);                // w^2 2^62
        const uint64_t t = mulhi1(mt, w2);               // m w^2 2^62, close to 2^62
        const uint64_t e = 0xC000000000000000ull - t;    // (3 - m w^2) 2^62, close to 2^63
        const uint64_t hi = mulhi1(y, e);                // w (3 - m w^2) 2^125 / 2^64
        y = (hi >> 63) ? ~0ull : (hi << 1);              // w' 2^63
    }
    {
        const uint64_t w2 = mulhi3(y, y);
        const uint64_t t = mulhi3(mt, w2);
        const uint64_t e = 0xC000000000000000ull - t;
        const uint64_t hi = mulhi3(y, e);
        y = (hi >> 63) ? ~0ull : (hi << 1);
    }
    *y_out = y;
    // sqrt(M) = m w 2^53 ~ mulhi(mt, y) / 2^10
    uint64_t q = mulhi3(mt, y) >> 10;
    int64_t r = (int64_t)(m_lo - q * q);                 // M - q^2, exact: |r| < 2^60
    if (r < 0) { q -= 1; r += (int64_t)(2 * q + 1); }
    if (r < 0) { q -= 1; r += (int64_t)(2 * q + 1); }
    if (r > (int64_t)(2 * q)) { r -= (int64_t)(2 * q + 1); q += 1; }
    if (r > (int64_t)(2 * q)) { r -= (int64_t)(2 * q + 1); q += 1; }
    // round to nearest: up iff M > (q + 1/2)^2, i.e. r > q (no ties exist)
    const bool up = r > (int64_t)q;
    const int fr = (f + 1022 + odd) >> 1;                // biased exponent of the root
    const double c = u2d(((uint64_t)(fr - 1) << 52) + q + (uint64_t)up);
    if (rem) {
        // a - c^2 = (M - Q^2) 2^(2 er - 104), Q the returned significand
        const int64_t rs = up ? r - (int64_t)(2 * q + 1) : r;
        uint64_t rb;
        if (pack_exact(rs, 2 * (fr - 1023) - 104, &rb)) *rem = u2d(rb);
        else *rem = native_fma(u2d(d2u(c) ^ kSign), c, a);
    }
    return c;
}

// 2 * c exactly as the IEEE multiplication, in integer form: an exponent
// increment for normal c, a doubled significand for subnormal c (which may
// carry into the smallest normal exponent), Inf from the top binade, and Inf,
// NaN and zeros unchanged.
TFS_HD double twice(double c) {
    const uint64_t u = d2u(c);
    const unsigned e = (unsigned)((u >> 52) & 0x7FF);
    const uint64_t sign = u & kSign;
    if (e - 1u < 2045u) return u2d(u + (1ull << 52));
    if (e == 0) return u2d(sign | ((u & kFrac) << 1));
    if (e == 2046) return u2d(sign | 0x7FF0000000000000ull);
    return c;
}

TFS_HD double native_mul(double a, double b) {
#if defined(__CUDA_ARCH__)
    double r;
    asm volatile("mul.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b));
    return r;
#else
    volatile double r = a * b;
    return r;
#endif
}

// The exact 106-bit product P = ma mb of two significands below 2^53 as
// (hi, lo) 64-bit words, from four 32 x 32-bit products: the high halves
// are below 2^21, so every partial sum stays below 2^64.
TFS_HD void mul53(uint64_t ma, uint64_t mb, uint64_t &hi, uint64_t &lo) {
    const uint64_t a0 = ma & 0xFFFFFFFFull, a1 = ma >> 32, b0 = mb & 0xFFFFFFFFull, b1 = mb >> 32;
    const uint64_t p00 = a0 * b0;
    const uint64_t mid = a0 * b1 + a1 * b0 + (p00 >> 32);   // < 2^54 + 2^32
    lo = (mid << 32) | (p00 & 0xFFFFFFFFull);
    hi = a1 * b1 + (mid >> 32);
}

// Correctly rounded a * b.  Normal operands whose product is normal (or
// overflows) run on the integer pipes: the 106-bit product of the
// significands, one normalisation step, round to nearest even on the
// guard bits plus a sticky bit; the carry of a rounded-up significand
// propagates into the exponent (and to Inf past the top binade) by the
// packing addition.  NaN, Inf and zero operands are resolved in integer
// form; subnormal operands and products near the underflow threshold go
// native.
TFS_HD double mul_rn(double a, double b) {
    const uint64_t ua = d2u(a), ub = d2u(b);
    const int fa = (int)((ua >> 52) & 0x7FF), fb = (int)((ub >> 52) & 0x7FF);
    const int e = fa + fb - 1023;                        // result field for a significand product in [1, 2)
    const uint64_t sign = (ua ^ ub) & kSign;
    if ((unsigned)(fa - 1) >= 2046u || (unsigned)(fb - 1) >= 2046u || e < 1 || e > 2046) {
        const uint64_t xa = ua & ~kSign, xb = ub & ~kSign, inf = 0x7FF0000000000000ull;
        if (xa > inf || xb > inf) return u2d(0x7FF8000000000000ull);
        if (xa == inf || xb == inf) return u2d((xa == 0 || xb == 0) ? 0x7FF8000000000000ull : (sign | inf));
        if (xa == 0 || xb == 0) return u2d(sign);
        if (e > 2046 && fa != 0 && fb != 0) return u2d(sign | inf);   // product >= 2^1024
        return native_mul(a, b);
    }
    uint64_t hi, lo;
    mul53((ua & kFrac) | kHid, (ub & kFrac) | kHid, hi, lo);   // P in [2^104, 2^106)
    const int top = (int)(hi >> 41);                     // product of significands in [2, 4)
    const int sh = 52 + top;                             // bits below the 53-bit significand
    uint64_t q = (hi << (12 - top)) | (lo >> sh);
    const uint64_t R = lo & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    q += (R > half) | ((R == half) & ((q & 1) != 0));
    const uint64_t r = ((uint64_t)(e + top - 1) << 52) + q, inf = 0x7FF0000000000000ull;
    return u2d(sign | (r >= inf ? inf : r));            // past the top binade: Inf
}

// Algorithm 3's pair from one integer product: p = RN(a b) and the exact
// error e = a b - p, bit-identical to a multiplication and fma(a, b, -p).
// The 106-bit product of the significands gives p by round to nearest even
// and e as its low part minus the rounding (exact whenever it is not
// subnormal; a zero error is +0, as the fused operation returns).  Zero,
// Inf and NaN operands are resolved in integer form; subnormal operands,
// products near either end of the range and errors below the normal range
// use the native pair.
TFS_HD void two_prod_rn(double a, double b, double &p, double &e) {
    const uint64_t ua = d2u(a), ub = d2u(b);
    const int fa = (int)((ua >> 52) & 0x7FF), fb = (int)((ub >> 52) & 0x7FF);
    const int ef = fa + fb - 1023;
    const uint64_t sign = (ua ^ ub) & kSign;
    if ((unsigned)(fa - 1) >= 2046u || (unsigned)(fb - 1) >= 2046u || ef < 111 || ef > 2044) {
        const uint64_t xa = ua & ~kSign, xb = ub & ~kSign, inf = 0x7FF0000000000000ull;
        const uint64_t nan = 0x7FF8000000000000ull;
        if (xa > inf || xb > inf) { p = u2d(nan); e = u2d(nan); return; }
        if (xa == inf || xb == inf) {
            p = u2d((xa == 0 || xb == 0) ? nan : (sign | inf));
            e = u2d(nan);
            return;
        }
        if (xa == 0 || xb == 0) { p = u2d(sign); e = 0.0; return; }
        p = native_mul(a, b);
        e = native_fma(a, b, u2d(d2u(p) ^ kSign));
        return;
    }
    const uint64_t ma = (ua & kFrac) | kHid, mb = (ub & kFrac) | kHid;
    uint64_t hi, lo;
    mul53(ma, mb, hi, lo);                               // P in [2^104, 2^106), hi in [2^40, 2^42)
    const int top = (int)(hi >> 41);                     // P >= 2^105
    const int sh = 52 + top;                             // bits below the 53-bit significand
    uint64_t q = (hi << (12 - top)) | (lo >> sh);       // P >> sh, in [2^52, 2^53)
    const uint64_t R = lo & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    const bool up = (R > half) | ((R == half) & ((q & 1) != 0));
    q += up;
    p = u2d(sign | (((uint64_t)(ef + top - 1) << 52) + q));
    // e = P - q 2^sh in units of 2^(ef-1127): R, or R - 2^sh after rounding
    // up; |e| <= 2^(sh-1)
    const int64_t ei = up ? (int64_t)R - (int64_t)(1ull << sh) : (int64_t)R;
    if (ei == 0) { e = 0.0; return; }
    const uint64_t se = sign ^ (ei < 0 ? kSign : 0);
    const uint64_t mag = (uint64_t)(ei < 0 ? -ei : ei);
    const int lz = clz64(mag);                           // >= 11: mag < 2^53
    const int lead = 63 - lz + ef - 1127;                // exponent of e's leading bit, >= -1016
    e = u2d(se | ((uint64_t)(lead + 1023) << 52) | ((mag << (lz - 11)) & kFrac));
}

// Correctly rounded a + b.  Normal operands run on the integer pipes: the
// significands aligned in 64-bit words with 10 guard bits, the bits shifted
// out of the smaller operand jammed into its lowest bit (sticky), exact
// addition or subtraction, normalisation, round to nearest even.  An exact
// zero sum is +0.  NaN, Inf and zero operands are resolved in integer form;
// subnormal operands and sums that land below the normal range go native.
TFS_HD double add_rn(double a, double b) {
    uint64_t ua = d2u(a), ub = d2u(b);
    uint64_t xa = ua & ~kSign, xb = ub & ~kSign;
    const uint64_t inf = 0x7FF0000000000000ull;
    int fa = (int)(xa >> 52), fb = (int)(xb >> 52);
    if ((unsigned)(fa - 1) >= 2046u || (unsigned)(fb - 1) >= 2046u) {
        if (xa > inf || xb > inf) return u2d(0x7FF8000000000000ull);
        if (xa == inf || xb == inf) {
            if (xa == inf && xb == inf && ((ua ^ ub) & kSign)) return u2d(0x7FF8000000000000ull);
            return xa == inf ? a : b;
        }
        if (xa == 0 && xb == 0) return u2d(ua & ub);      // -0 only when both are -0
        if (xb == 0 && fa != 0) return a;
        if (xa == 0 && fb != 0) return b;
        return native_add(a, b);
    }
    if (xa < xb) {                                       // a: the larger magnitude
        uint64_t t = ua; ua = ub; ub = t;
        t = xa; xa = xb; xb = t;
        int f = fa; fa = fb; fb = f;
    }
    const uint64_t sign = ua & kSign;
    const int d = fa - fb;
    const uint64_t mbig = ((xa & kFrac) | kHid) << 10;  // leading bit at 62
    uint64_t msml = ((xb & kFrac) | kHid) << 10;
    if (d >= 64) msml = 1;                               // only the sticky bit remains
    else if (d > 0) msml = (msml >> d) | (uint64_t)((msml << (64 - d)) != 0);
    int e = fa;
    uint64_t m;
    if ((ua ^ ub) & kSign) {
        m = mbig - msml;
        if (m == 0) return 0.0;
        const int lz = clz64(m) - 1;                     // shift the leading bit back to 62
        e -= lz;
        if (e < 1) return native_add(a, b);              // result below the normal range
        m <<= lz;
    } else {
        m = mbig + msml;
        if (m >> 63) { m = (m >> 1) | (m & 1); e += 1; }
    }
    uint64_t q = m >> 10;
    const uint64_t rem = m & 0x3FF;
    q += (rem > 0x200) | ((rem == 0x200) & (q & 1));
    const uint64_t r = ((uint64_t)(e - 1) << 52) + q;   // may carry to the Inf pattern
    return u2d(sign | (r >= inf ? inf : r));
}

// sqrt(u) correctly rounded, given yx = the reciprocal root that
// sqrt_rn_y(x) returned for a nearby x (RTF1 takes the root of x0 and of
// u0 = RN(x0 + x1), usually a few ulps apart).  When u and x share the
// binade and their significands differ by at most 2^8 units, yx is within
// 2^-44 of u's reciprocal root: the root estimate is within 2^9 units, one
// remainder-driven step brings it within two units, and the exact integer
// remainder finishes as in sqrt_rn_y.  Otherwise the full routine runs.
// With rem != nullptr, *rem also receives RN(u - v^2) for the returned root
// v, the bits of fma(-v, v, u) (Algorithm 5's exact residual).
// The general case of sqrt_rn_near (u far from x, or a special value):
// the full root, and its residual where rem is wanted.
TFS_COLD double sqrt_near_general(double u, double *rem, uint64_t *y_out) {
    const uint64_t uu = d2u(u);
    uint64_t y;
    const double v = sqrt_rn_y(u, &y);
    if (y_out) *y_out = y;
    if (rem) {
        // fma(-v, v, u) without a native operation where the root is NaN
        // (NaN), +Inf (-Inf + Inf: NaN) or a zero (v = u, -u u + u = u)
        const uint64_t xu = uu & ~kSign, inf = 0x7FF0000000000000ull;
        if ((uu >> 63 && xu != 0) || xu >= inf) *rem = u2d(0x7FF8000000000000ull);
        else if (xu == 0) *rem = u;
        else *rem = native_fma(u2d(d2u(v) ^ kSign), v, u);
    }
    return v;
}

// With y_out != nullptr, *y_out receives a reciprocal estimate for dividing
// by 2 v (the divisor RTF1's RPF1 step takes) that div_rn_y accepts: on the
// near path, yx lowered by 2^-44 relative (v and sqrt(x) share the binade
// and differ by at most 2^-45 relative, and yx is within 2^-52 of the
// reciprocal of sqrt(x)'s significand, so the lowered value is never above
// the reciprocal of v's significand and at most 1.5 2^-44 below it); on the
// general path, the full root's own estimate; 0 (no estimate) for a NaN root.
TFS_HD double sqrt_rn_near(double u, double x, uint64_t yx, double *rem = nullptr, uint64_t *y_out = nullptr) {
    const uint64_t uu = d2u(u), ux = d2u(x);
    // a negative radicand or a NaN with the sign bit set: NaN root and
    // residual, resolved here because they are common (a chain whose value
    // went negative) while the general case below is rare
    if ((uu >> 63) && (uu << 1)) {
        if (rem) *rem = u2d(0x7FF8000000000000ull);
        if (y_out) *y_out = 0;
        return u2d(0x7FF8000000000000ull);
    }
    const int f = (int)(uu >> 52);
    const uint64_t mu = (uu & kFrac) | kHid, mx = (ux & kFrac) | kHid;
    const uint64_t diff = mu > mx ? mu - mx : mx - mu;
    if (yx == 0 || f != (int)(ux >> 52) || (unsigned)(f - 1) >= 2046u || diff > 256)
        return sqrt_near_general(u, rem, y_out);
    if (y_out) *y_out = yx - (yx >> 44);
    const int odd = f & 1;
    const int s = odd ? 52 : 53;
    const uint64_t m_hi = mu >> (64 - s), m_lo = mu << s;
    const uint64_t mt = (m_hi << 22) | (m_lo >> 42);
    // the estimate is within 257 units of Q; 260 below it, the remainder
    // M - q^2 lies in [0, 2^63.02) and is exact modulo 2^64
    uint64_t q = (mulhi3(mt, yx) >> 10) - 260;
    uint64_t r = m_lo - q * q;
    // dq ~ r / (2 q) = r w / 2^54 / ... = mulhi(r, yx) / 2^53 (high words: low
    // by under 2^-20 units)
    const uint64_t dq = mulhi1(r, yx) >> 53;
    q += dq;
    int64_t rr = (int64_t)(m_lo - q * q);                 // |M - q^2| < 2^60 now
    if (rr < 0) { q -= 1; rr += (int64_t)(2 * q + 1); }
    if (rr < 0) { q -= 1; rr += (int64_t)(2 * q + 1); }
    if (rr > (int64_t)(2 * q)) { rr -= (int64_t)(2 * q + 1); q += 1; }
    if (rr > (int64_t)(2 * q)) { rr -= (int64_t)(2 * q + 1); q += 1; }
    const bool up = rr > (int64_t)q;
    const int fr = (f + 1022 + odd) >> 1;
    const double v = u2d(((uint64_t)(fr - 1) << 52) + q + (uint64_t)up);
    if (rem) {
        // u - v^2 = (M - Q^2) 2^(2 er - 104), Q the returned significand
        const int64_t rs = up ? rr - (int64_t)(2 * q + 1) : rr;
        uint64_t rb;
        if (pack_exact(rs, 2 * (fr - 1023) - 104, &rb)) *rem = u2d(rb);
        else *rem = native_fma(u2d(d2u(v) ^ kSign), v, u);
    }
    return v;
}

// RN(|z| 2^k) as bits for an integer k <= 0 (the scaling of a panic
// threshold that is a power of two), exact for results in the normal range,
// round to nearest even into the subnormal range, Inf and NaN kept.
TFS_HD uint64_t scale_abs_pow2(uint64_t uz, int k) {
    const uint64_t a = uz & ~kSign;
    const int f = (int)(a >> 52);
    if (f == 0x7FF || a == 0) return a;
    if (f + k >= 1) return a + ((uint64_t)(int64_t)k << 52);   // stays normal: exponent shift
    // subnormal result: significand (with hidden bit when normal) >> (1 - f - k), or >> -k
    const uint64_t m = f ? ((a & kFrac) | kHid) : a;
    const int sh = f ? (1 - f - k) : -k;
    if (sh >= 64) return 0;
    const uint64_t q = m >> sh, rem = m & ((1ull << sh) - 1), half = sh ? (1ull << (sh - 1)) : 0;
    return q + ((rem > half) | ((rem == half) & (q & 1) & (sh > 0)));
}

// Signed integer significand m and scale q of a finite x = m 2^q.
TFS_HD void unpack(uint64_t u, int64_t &m, int &q) {
    const int e = (int)((u >> 52) & 0x7FF);
    const uint64_t f = (u & kFrac) | (e ? kHid : 0);
    q = (e ? e : 1) - 1075;
    m = (u >> 63) ? -(int64_t)f : (int64_t)f;
}

// m 2^sh modulo 2^64 for 0 <= sh; a shift of 64 or more gives 0.
TFS_HD uint64_t shl_mod(int64_t m, int sh) { return sh >= 64 ? 0 : ((uint64_t)m << sh); }

// The tail of Algorithm 1.2 (Two-Sum) by its six native operations.
TFS_HD double literal_sum_err(double a, double b, double s) {
#if defined(__CUDA_ARCH__)
    double t;
    asm volatile(
        "{\n\t.reg .f64 bv, av, ar, br;\n\t"
        "sub.rn.f64 bv, %3, %1;\n\t"
        "sub.rn.f64 av, %3, bv;\n\t"
        "sub.rn.f64 ar, %1, av;\n\t"
        "sub.rn.f64 br, %2, bv;\n\t"
        "add.rn.f64 %0, ar, br;\n\t}"
        : "=d"(t) : "d"(a), "d"(b), "d"(s));
    return t;
#else
    volatile double bv = s - a;
    volatile double av = s - bv;
    volatile double ar = a - av;
    volatile double br = b - bv;
    volatile double t = ar + br;
    return t;
#endif
}

// t = a + b - s exactly, where s = RN(a + b): bit-identical to the tail of
// Algorithm 1.2 (Two-Sum), whose result is +0 when the error is zero.  When
// both operands are below 2^1022 in magnitude no intermediate of the
// literal sequence can overflow and its tail is the exact error; otherwise
// (near-overflow operands, Inf, NaN) the literal sequence runs natively.
// All three of a, b, s are integer multiples of 2^qmin, the finer of the two
// operands' ulps, and |t| <= ulp(s)/2, so the integer A + B - S is small and
// is formed modulo 2^64 when the exponent gap is at most 60.  With a larger
// gap the smaller operand is below a quarter ulp of the larger: s is the
// larger operand and t the smaller one.
TFS_HD uint64_t sum_err_bits(uint64_t ua, uint64_t ub, uint64_t us);

TFS_HD double sum_err(double a, double b, double s) { return u2d(sum_err_bits(d2u(a), d2u(b), d2u(s))); }

// The same on bit patterns (so that a caller can negate an operand by its
// sign bit without the compiler forming a floating-point negation).
TFS_HD uint64_t sum_err_bits(uint64_t ua, uint64_t ub, uint64_t us) {
    const unsigned fa = (unsigned)((ua >> 52) & 0x7FF), fb = (unsigned)((ub >> 52) & 0x7FF);
    if ((fa >= 2045) | (fb >= 2045)) {
        // an Inf or NaN operand makes every variant of the literal sequence NaN
        if ((fa == 0x7FF) | (fb == 0x7FF)) return 0x7FF8000000000000ull;
        return d2u(literal_sum_err(u2d(ua), u2d(ub), u2d(us)));
    }
    int64_t ma, mb, ms;
    int qa, qb, qs;
    unpack(ua, ma, qa);
    unpack(ub, mb, qb);
    unpack(us, ms, qs);
    const int qmin = qa < qb ? qa : qb;
    const int gap = (qa > qb ? qa : qb) - qmin;
    if (gap > 60) {
        // t = the operand with the finer ulp (never -0: a zero error is +0)
        const uint64_t small = qa < qb ? ua : ub;
        return (small << 1) ? small : 0;
    }
    int64_t big = (int64_t)(shl_mod(ma, qa - qmin) + shl_mod(mb, qb - qmin));
    // s is a multiple of 2^qmin; its own scale may be finer when the sum cancels
    const int ds = qs - qmin;
    int64_t sv = ds >= 0 ? (int64_t)shl_mod(ms, ds) : (ms >> (-ds));
    const int64_t t = big - sv;
    if (t == 0) return 0;
    const uint64_t sign = t < 0 ? kSign : 0;
    const uint64_t mag = (uint64_t)(t < 0 ? -t : t);
    const int lz = clz64(mag);
    const int lead = 63 - lz + qmin;                     // exponent of the leading bit
    if (lead >= -1022) {
        const uint64_t frac = ((mag << lz) >> 11) & kFrac;   // exact: t fits 53 bits
        return sign | ((uint64_t)(lead + 1023) << 52) | frac;
    }
    return sign | (mag << (qmin + 1074));               // subnormal tail
}

// The tail of Algorithm 2.2 (Two-Diff) of a - b, d = RN(a - b), for
// operands that are usually close: when a and b are finite with the same
// sign and the same exponent field, b/2 <= a <= 2b (or both are subnormal),
// so a - b is exact (Sterbenz) and every step of the sequence is exact: the
// tail is +0.  Otherwise the general tail (sum_err_bits of a, -b, d).
TFS_HD uint64_t diff_err_near_bits(uint64_t ua, uint64_t ub, uint64_t ud) {
    if (((ua ^ ub) >> 52) == 0 && ((ua >> 52) & 0x7FF) != 0x7FF) return 0;
    return sum_err_bits(ua, ub ^ kSign, ud);
}

}  // namespace soft
}  // namespace tf
