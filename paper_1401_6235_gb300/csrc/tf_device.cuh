// Device-side twofold arithmetic (Latkin, "Twofold fast arithmetic").
//
// Every binary64 operation is either an explicit round-to-nearest intrinsic
// (__dadd_rn, __dsub_rn, __dmul_rn, __fma_rn), which the compiler never
// contracts or reassociates (the library is also built with -fmad=false), or
// an integer-pipe routine of tf_soft.cuh that returns the same bits as the
// IEEE operation (division, square root, the exact Two-Sum tail).  Each
// function performs the operations of its algorithm in the paper's order, so
// results are bit-identical to any correct implementation of the sequence.
#pragma once
#if !defined(__CUDACC_RTC__)
#include <cstdint>
#endif

#include "tf_soft.cuh"

namespace tf {

struct d2 { double z0, z1; };

// ------------------------------------------------------------------ bits
// (opaque moves, see soft::d2u: sign work on the bits stays on the integer pipes)
__device__ __forceinline__ uint64_t bits_of(double v) { return soft::d2u(v); }
__device__ __forceinline__ double from_bits(uint64_t b) { return soft::u2d(b); }
__device__ __forceinline__ bool finite_bits(double v) {
    return ((bits_of(v) >> 52) & 0x7FF) != 0x7FF;
}

// ------------------------------------------------- Background: exact transforms

// Algorithm 1.2 (Two-Sum): a + b -> s + t, t the exact rounding error.
// s is one native addition; the tail t comes from soft::sum_err, which gives
// the bits of steps (2)-(6) (exact error, +0 when zero, the literal sequence
// near overflow and for Inf/NaN) on the integer pipes.
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &t) {
    s = __dadd_rn(a, b);
    t = soft::sum_err(a, b, s);
}

// Algorithm 1.2's result by Algorithm 1.1 on ordered operands: s = a + b,
// then the Fast-Two-Sum tail small - (s - big) with big the operand of the
// larger exponent field, which is the exact error (both subtractions are
// exact when the exponent of big is at least that of small, gradual
// underflow included); a zero error becomes +0, as Algorithm 1.2 returns.
// Operands at or near the overflow threshold, Inf and NaN take the integer
// tail (which follows the literal sequence there).  Two FP64 subtractions
// and a few integer instructions in place of the integer tail's ~80: for
// kernels whose integer pipes are busier than their FP64 pipe.
__device__ __forceinline__ void two_sum_fp(double a, double b, double &s, double &t) {
    s = __dadd_rn(a, b);
    const uint64_t ua = bits_of(a), ub = bits_of(b);
    const unsigned fa = (unsigned)(ua >> 52) & 0x7FF, fb = (unsigned)(ub >> 52) & 0x7FF;
    if ((fa >= 2045) | (fb >= 2045)) {
        t = soft::sum_err(a, b, s);
        return;
    }
    const bool sw = fb > fa;
    const double big = sw ? b : a, small = sw ? a : b;
    const uint64_t ut = bits_of(__dsub_rn(small, __dsub_rn(s, big)));
    t = from_bits((ut << 1) ? ut : 0);
}

// Algorithm 2.2 (Two-Diff): a - b -> d + t.  Steps (4),(5) in Shewchuk's
// order (b# = b' - b, a# = a - a'), which makes a - b = d + t exact.  With
// round-to-nearest every step of Two-Diff(a, b) is the negation-mirror of
// Two-Sum(a, -b) (b' = a - d = -(d - a), a' = b' + d = d - (d - a), ...), so
// its tail is the Two-Sum tail of (a, -b, d), bit for bit.
__device__ __forceinline__ void two_diff(double a, double b, double &d, double &t) {
    d = __dsub_rn(a, b);
    // -b by its sign bit, handed over as a bit pattern
    t = from_bits(soft::sum_err_bits(bits_of(a), bits_of(b) ^ 0x8000000000000000ull, bits_of(d)));
}

// Algorithm 3 (Two-Product-FMA): p = a*b, e = fma(a, b, -p); both from one
// integer product (soft::two_prod_rn, the same bits as the two native ops).
__device__ __forceinline__ void two_prod(double a, double b, double &p, double &e) {
    soft::two_prod_rn(a, b, p, e);
}

// Correctly rounded division and square root (integer pipes, IEEE bits).
__device__ __forceinline__ double div_rn(double a, double b) { return soft::div_rn(a, b); }
__device__ __forceinline__ double sqrt_rn(double a) { return soft::sqrt_rn(a); }

// 2 * c with IEEE bits, in integer form (soft::twice).
__device__ __forceinline__ double twice(double c) { return soft::twice(c); }

// Algorithm 4: q = a/b, r = fma(-q, b, a) = a - q b exactly.
__device__ __forceinline__ void div_rem(double a, double b, double &q, double &r) {
    q = div_rn(a, b);
    r = __fma_rn(-q, b, a);
}

// Algorithm 5: c = sqrt(a), d = fma(-c, c, a) = a - c^2 exactly.
__device__ __forceinline__ void sqrt_rem(double a, double &c, double &d) {
    c = sqrt_rn(a);
    d = __fma_rn(-c, c, a);
}

// ----------------------------------------------------------- Algorithms

// ATF1: z0 = x0 + y0; z1 = (x1 + y1) + err(x0 + y0).
__device__ __forceinline__ d2 atf1(double x0, double x1, double y0, double y1) {
    double s, e;
    two_sum(x0, y0, s, e);
    return {s, __dadd_rn(__dadd_rn(x1, y1), e)};
}

// ATF1 with the Two-Sum tail from two_sum_fp (same bits; fewer integer
// instructions for two more FP64 ones).
__device__ __forceinline__ d2 atf1_fp(double x0, double x1, double y0, double y1) {
    double s, e;
    two_sum_fp(x0, y0, s, e);
    return {s, __dadd_rn(__dadd_rn(x1, y1), e)};
}

// ATF1.1: z0 = x0 + y0; z1 = x1 + err(x0 + y0).
__device__ __forceinline__ d2 atf11(double x0, double x1, double y0) {
    double s, e;
    two_sum(x0, y0, s, e);
    return {s, __dadd_rn(x1, e)};
}

// STF1: z0 = x0 - y0; z1 = (x1 - y1) + err(x0 - y0).
__device__ __forceinline__ d2 stf1(double x0, double x1, double y0, double y1) {
    double d, e;
    two_diff(x0, y0, d, e);
    return {d, __dadd_rn(__dsub_rn(x1, y1), e)};
}

// STF1.1: z0 = x0 - y0; z1 = x1 + err(x0 - y0).
__device__ __forceinline__ d2 stf11(double x0, double x1, double y0) {
    double d, e;
    two_diff(x0, y0, d, e);
    return {d, __dadd_rn(x1, e)};
}

// MTF1: z0 = p00; z1 = (e00 + p11) + (p01 + p10).
__device__ __forceinline__ d2 mtf1(double x0, double x1, double y0, double y1) {
    double p00, e00;
    two_prod(x0, y0, p00, e00);
    double p11 = __dmul_rn(x1, y1);
    double p01 = __dmul_rn(x0, y1);
    double p10 = __dmul_rn(x1, y0);
    return {p00, __dadd_rn(__dadd_rn(e00, p11), __dadd_rn(p01, p10))};
}

// MTF1.1: z0 = p00; z1 = e00 + p10.
__device__ __forceinline__ d2 mtf11(double x0, double x1, double y0) {
    double p00, e00;
    two_prod(x0, y0, p00, e00);
    return {p00, __dadd_rn(e00, __dmul_rn(x1, y0))};
}

// The divisions below share reciprocal estimates (soft::div_rn_y): both
// divisions of DTF1.1 / DTF1.1.1 divide by y0; DTF1's second divisor
// d0 = y0 (+) y1 usually rounds back to y0; RPF1's divisor 2 z0 has the
// significand of z0, whose reciprocal square-root estimate the square root
// already produced.  Every quotient is still the correctly rounded one.

// The remainder fma(-z0, y0, x0) of Algorithm 4 comes packed from the
// integer division's own exact remainder (soft::div_rn_y, same bits).

// DTF1.1.1: z0 = x0/y0; r1 = fma(-z0, y0, x0); z1 = r1/y0.
__device__ __forceinline__ d2 dtf111(double x0, double y0) {
    const uint64_t yb = soft::recip_of(y0);
    double r;
    const double q = soft::div_rn_y(x0, y0, yb, &r);
    return {q, soft::div_rn_y(r, y0, yb)};
}

// DTF1.1: z0 = x0/y0; r = fma(-z0, y0, x0); c = r + x1; z1 = c/y0.
__device__ __forceinline__ d2 dtf11(double x0, double x1, double y0) {
    const uint64_t yb = soft::recip_of(y0);
    double r;
    const double q = soft::div_rn_y(x0, y0, yb, &r);
    return {q, soft::div_rn_y(__dadd_rn(r, x1), y0, yb)};
}

// DTF1: z0 = x0/y0; r0 = fma(-z0, y0, x0); r1 = fma(-z0, y1, x1);
//       c0 = r0 + r1; d0 = y0 + y1; z1 = c0/d0.
__device__ __forceinline__ d2 dtf1(double x0, double x1, double y0, double y1) {
    const uint64_t yb = soft::recip_of(y0);
    double r0;
    const double q = soft::div_rn_y(x0, y0, yb, &r0);
    const double r1 = __fma_rn(-q, y1, x1);
    const double c0 = __dadd_rn(r0, r1);
    const double d0 = __dadd_rn(y0, y1);
    uint64_t yd = yb;
    if (bits_of(d0) != bits_of(y0)) yd = soft::recip_of(d0);
    return {q, soft::div_rn_y(c0, d0, yd)};
}

// The residual fma(-z0, z0, x0) of Algorithm 5 comes packed from the integer
// root's own exact remainder (soft::sqrt_rn_y, same bits).

// RPF1: z0 = sqrt(x0); z1 = (x1 + fma(-z0, z0, x0)) / (2 z0).
__device__ __forceinline__ d2 rpf1(double x0, double x1) {
    uint64_t y;
    double d;
    const double c = soft::sqrt_rn_y(x0, &y, &d);
    return {c, soft::div_rn_y(__dadd_rn(x1, d), twice(c), y)};
}

// RPF1.1: z0 = sqrt(x0); z1 = fma(-z0, z0, x0) / (2 z0).
__device__ __forceinline__ d2 rpf11(double x0) {
    uint64_t y;
    double d;
    const double c = soft::sqrt_rn_y(x0, &y, &d);
    return {c, soft::div_rn_y(d, twice(c), y)};
}

// RTF1: z0 = sqrt(x0); (u0,u1) = Two-Sum(x0, x1); (v0,v1) = RPF1(u0,u1);
//       (w0,w1) = STF1.1((v0,v1), z0); z1 = w0 + w1.
// The root of u0 (a few ulps from x0) starts from the reciprocal root that
// the root of x0 produced (soft::sqrt_rn_near; same correctly rounded bits),
// and RPF1's division by 2 v0 reuses that estimate.  v0 and z0 are roots of
// nearby values, so STF1.1's difference v0 - z0 is usually exact and its
// tail +0 without the general Two-Diff tail (soft::diff_err_near_bits).
// (A short cut for u0 = x0 that reused z0's root and residual measured
// slower on the chain workload: enough lanes of a warp have tails that move
// the head for the warp to run both paths.)
__device__ __forceinline__ d2 rtf1(double x0, double x1) {
    uint64_t yz;
    const double z0 = soft::sqrt_rn_y(x0, &yz);
    double u0, u1;
    two_sum_fp(x0, x1, u0, u1);
    double d;                                                // fma(-v0, v0, u0), packed
    uint64_t yv;
    const double v0 = soft::sqrt_rn_near(u0, x0, yz, &d, &yv);   // RPF1 on (u0, u1)
    const double v1 = soft::div_rn_y(__dadd_rn(u1, d), twice(v0), yv);
    const double w0 = __dsub_rn(v0, z0);                     // STF1.1((v0, v1), z0)
    const double w1 = __dadd_rn(v1, from_bits(soft::diff_err_near_bits(bits_of(v0), bits_of(z0), bits_of(w0))));
    return {z0, __dadd_rn(w0, w1)};
}

// -------------------------------------------- coupled (Dekker emulation)

// Algorithm 1.1 (Fast Two-Sum), its three operations taken literally: the
// renormalisation of a twofold (exact when |a| >= |b|).
__device__ __forceinline__ d2 fast_two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    const double bv = __dsub_rn(s, a);
    return {s, __dsub_rn(b, bv)};
}
__device__ __forceinline__ d2 renorm(d2 z) { return fast_two_sum(z.z0, z.z1); }

// MPF1 (coupled x, y): z0 = p00;  z1 = e00 + (p01 + p10)  (p11 omitted).
__device__ __forceinline__ d2 mpf1(double x0, double x1, double y0, double y1) {
    double p00, e00;
    two_prod(x0, y0, p00, e00);
    const double p01 = __dmul_rn(x0, y1);
    const double p10 = __dmul_rn(x1, y0);
    return {p00, __dadd_rn(e00, __dadd_rn(p01, p10))};
}

// DPF1 (coupled x, y): z0 = x0/y0; r0 = fma(-z0, y0, x0); r1 = fma(-z0, y1, x1);
//       c0 = r0 + r1; z1 = c0/y0  (both divisions by y0 share one reciprocal).
__device__ __forceinline__ d2 dpf1(double x0, double x1, double y0, double y1) {
    const uint64_t yb = soft::recip_of(y0);
    double r0;
    const double q = soft::div_rn_y(x0, y0, yb, &r0);
    const double r1 = __fma_rn(-q, y1, x1);
    return {q, soft::div_rn_y(__dadd_rn(r0, r1), y0, yb)};
}

// ------------------------------------------------------- operand kinds
// Operand kinds: (twofold, twofold) general; (twofold, dotted) ".1";
// (dotted, twofold) general with x1 = +0; (dotted, dotted) exact transform
// or DTF1.1.1; sqrt of dotted: RPF1.1.
enum Op : int { OP_ADD = 1, OP_SUB = 2, OP_MUL = 3, OP_DIV = 4, OP_SQRT = 5,
               OP_PADD = 6, OP_PSUB = 7, OP_PMUL = 8, OP_PDIV = 9, OP_PSQRT = 10 };

__device__ __forceinline__ d2 apply(int op, double x0, double x1, bool xd, double y0, double y1,
                                    bool yd) {
    if (op == OP_SQRT) return xd ? rpf11(x0) : rtf1(x0, x1);
    if (xd && yd) {
        d2 z;
        switch (op) {
        case OP_ADD: two_sum(x0, y0, z.z0, z.z1); return z;
        case OP_SUB: two_diff(x0, y0, z.z0, z.z1); return z;
        case OP_MUL: two_prod(x0, y0, z.z0, z.z1); return z;
        default: return dtf111(x0, y0);
        }
    }
    if (yd) {
        switch (op) {
        case OP_ADD: return atf11(x0, x1, y0);
        case OP_SUB: return stf11(x0, x1, y0);
        case OP_MUL: return mtf11(x0, x1, y0);
        default: return dtf11(x0, x1, y0);
        }
    }
    if (xd) x1 = 0.0;
    switch (op) {
    // ATF1 of two twofolds with the floating-point Two-Sum tail (same
    // bits): in elementwise programs the integer pipes are the busier ones
    // (the divisions and roots run there), and on the chain program this
    // form measured 3 % faster (11.61 against 11.97 ms at 2^28)
    case OP_ADD: return atf1_fp(x0, x1, y0, y1);
    case OP_SUB: return stf1(x0, x1, y0, y1);
    case OP_MUL: return mtf1(x0, x1, y0, y1);
    default: return dtf1(x0, x1, y0, y1);
    }
}

// Coupled ("p") operations, op = OP_PADD .. OP_PSQRT: the coupled variant of
// the operand kinds, then Fast Two-Sum renormalisation; with every operand
// dotted the output is already coupled and is returned as is.
__device__ __forceinline__ d2 apply_coupled(int op, double x0, double x1, bool xd, double y0, double y1,
                                            bool yd) {
    const int base = op - 5;
    if (base == OP_SQRT) return xd ? rpf11(x0) : renorm(rpf1(x0, x1));
    if (xd && yd) return apply(base, x0, x1, true, y0, y1, true);
    if (yd) {
        switch (base) {
        case OP_ADD: return renorm(atf11(x0, x1, y0));
        case OP_SUB: return renorm(stf11(x0, x1, y0));
        case OP_MUL: return renorm(mtf11(x0, x1, y0));         // MPF1.1 = MTF1.1
        default: return renorm(dtf11(x0, x1, y0));             // DPF1.1 = DTF1.1
        }
    }
    if (xd) x1 = 0.0;
    switch (base) {
    case OP_ADD: return renorm(atf1(x0, x1, y0, y1));
    case OP_SUB: return renorm(stf1(x0, x1, y0, y1));
    case OP_MUL: return renorm(mpf1(x0, x1, y0, y1));
    default: return renorm(dpf1(x0, x1, y0, y1));
    }
}

// Any operation; P: the program contains coupled operations (kernels without
// them do not carry their code).
template <bool P>
__device__ __forceinline__ d2 apply_any(int op, double x0, double x1, bool xd, double y0, double y1, bool yd) {
    if (P && op > OP_SQRT) return apply_coupled(op, x0, x1, xd, y0, y1, yd);
    return apply(op, x0, x1, xd, y0, y1, yd);
}

__device__ __forceinline__ bool unary(int op) { return op == OP_SQRT || op == OP_PSQRT; }

// Plain binary64 operation (the "dotted" arithmetic the twofold shadows).
__device__ __forceinline__ double apply_plain(int op, double a, double b) {
    if (op > OP_SQRT) op -= 5;      // the plain twin of a coupled op is the basic op
    switch (op) {
    case OP_ADD: return __dadd_rn(a, b);
    case OP_SUB: return __dsub_rn(a, b);
    case OP_MUL: return __dmul_rn(a, b);
    case OP_DIV: return __ddiv_rn(a, b);
    default: return __dsqrt_rn(a);
    }
}

// The same plain operation with the division and square root on the integer
// pipes (soft::div_rn / soft::sqrt_rn: correctly rounded, the same bits).
__device__ __forceinline__ double apply_plain_int(int op, double a, double b) {
    if (op > OP_SQRT) op -= 5;
    if (op == OP_DIV) return soft::div_rn(a, b);
    if (op == OP_SQRT) return soft::sqrt_rn(a);
    return apply_plain(op, a, b);
}

// ---------------------------------------------------------- panic flag
struct FlagCfg {
    int mode;      // 0 REL, 1 ULP
    double tau;    // REL threshold
    double m;      // ULP threshold
    int k;         // REL: tau = 2^k exactly (k <= 0), else 1 (use the multiplication)
};

// ulp(v) = 2^(max(e,-1022)-52) from the exponent field; NaN for Inf/NaN.
__device__ __forceinline__ double ulp_of(double v) {
    int e = (int)((bits_of(v) >> 52) & 0x7FF);
    if (e == 0x7FF) return from_bits(0x7FF8000000000000ull);
    if (e == 0) e = 1;
    int p = e - 1075;                       // exponent of the ulp, >= -1074
    if (p >= -1022) return from_bits((uint64_t)(p + 1023) << 52);
    return from_bits(1ull << (p + 1074));   // subnormal power of two
}

// |z1| > lim compared on the integer pipe: for non-negative non-NaN
// binary64 values the bit patterns order like the values; a NaN on either
// side compares false, as the floating-point comparison does.
__device__ __forceinline__ uint8_t flag_of(double z0, double z1, const FlagCfg &f) {
    uint8_t r = 0;
    if (!finite_bits(z0) || !finite_bits(z1)) r |= 2;
    // tau >= 0, so |RN(tau z0)| = RN(tau |z0|): the magnitude is taken on the
    // bits; a power-of-two tau (the default 2^-40) scales in integer form
    uint64_t l;
    if ((f.mode & 3) == 0) {
        if (f.k <= 0) l = soft::scale_abs_pow2(bits_of(z0), f.k);
        else l = bits_of(__dmul_rn(f.tau, z0)) & 0x7FFFFFFFFFFFFFFFull;
    } else {
        l = bits_of(__dmul_rn(f.m, ulp_of(z0))) & 0x7FFFFFFFFFFFFFFFull;
    }
    const uint64_t a = bits_of(z1) & 0x7FFFFFFFFFFFFFFFull;
    const uint64_t inf = 0x7FF0000000000000ull;
    if (a <= inf && l <= inf && a > l) r |= 1;
    return r;
}

}  // namespace tf
