// Device-side twofold arithmetic over binary32 (the paper's algorithms are
// generic over the number type; its logs print float and double rows).
//
// Every operation is an explicit round-to-nearest binary32 intrinsic
// (__fadd_rn, __fsub_rn, __fmul_rn, __fmaf_rn, __fdiv_rn, __fsqrt_rn), which
// the compiler never contracts or reassociates and which keep subnormals
// (the library is built without flush-to-zero).  The FP32 pipe is the widest
// on this GPU, so the exact transforms are the literal operation sequences.
// The functions overload the binary64 ones of tf_device.cuh by argument type.
#pragma once
#if !defined(__CUDACC_RTC__)
#include <cstdint>
#endif

#include "tf_device.cuh"

namespace tf {

struct f2 { float z0, z1; };

// Algorithm 1.2 (Two-Sum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &t) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    const float bs = __fsub_rn(b, bv);
    const float as = __fsub_rn(a, av);
    t = __fadd_rn(as, bs);
}

// Algorithm 2.2 (Two-Diff) in Shewchuk's order: b# = b' - b, a# = a - a'.
__device__ __forceinline__ void two_diff(float a, float b, float &d, float &t) {
    d = __fsub_rn(a, b);
    const float bv = __fsub_rn(a, d);
    const float av = __fadd_rn(bv, d);
    const float bs = __fsub_rn(bv, b);
    const float as = __fsub_rn(a, av);
    t = __fadd_rn(as, bs);
}

// Algorithm 3 (Two-Product with FMA).
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Algorithms 4 and 5: exact remainder and residual.
__device__ __forceinline__ void div_rem(float a, float b, float &q, float &r) {
    q = __fdiv_rn(a, b);
    r = __fmaf_rn(-q, b, a);
}
__device__ __forceinline__ void sqrt_rem(float a, float &c, float &d) {
    c = __fsqrt_rn(a);
    d = __fmaf_rn(-c, c, a);
}

__device__ __forceinline__ f2 atf1(float x0, float x1, float y0, float y1) {
    float s, e;
    two_sum(x0, y0, s, e);
    return {s, __fadd_rn(__fadd_rn(x1, y1), e)};
}
__device__ __forceinline__ f2 atf11(float x0, float x1, float y0) {
    float s, e;
    two_sum(x0, y0, s, e);
    return {s, __fadd_rn(x1, e)};
}
__device__ __forceinline__ f2 stf1(float x0, float x1, float y0, float y1) {
    float d, e;
    two_diff(x0, y0, d, e);
    return {d, __fadd_rn(__fsub_rn(x1, y1), e)};
}
__device__ __forceinline__ f2 stf11(float x0, float x1, float y0) {
    float d, e;
    two_diff(x0, y0, d, e);
    return {d, __fadd_rn(x1, e)};
}
// MTF1: z1 = (e00 + p11) + (p01 + p10).
__device__ __forceinline__ f2 mtf1(float x0, float x1, float y0, float y1) {
    float p00, e00;
    two_prod(x0, y0, p00, e00);
    const float p11 = __fmul_rn(x1, y1), p01 = __fmul_rn(x0, y1), p10 = __fmul_rn(x1, y0);
    return {p00, __fadd_rn(__fadd_rn(e00, p11), __fadd_rn(p01, p10))};
}
__device__ __forceinline__ f2 mtf11(float x0, float x1, float y0) {
    float p00, e00;
    two_prod(x0, y0, p00, e00);
    return {p00, __fadd_rn(e00, __fmul_rn(x1, y0))};
}
// MPF1 (coupled): z1 = e00 + (p01 + p10).
__device__ __forceinline__ f2 mpf1(float x0, float x1, float y0, float y1) {
    float p00, e00;
    two_prod(x0, y0, p00, e00);
    return {p00, __fadd_rn(e00, __fadd_rn(__fmul_rn(x0, y1), __fmul_rn(x1, y0)))};
}
__device__ __forceinline__ f2 dtf111(float x0, float y0) {
    float q, r;
    div_rem(x0, y0, q, r);
    return {q, __fdiv_rn(r, y0)};
}
__device__ __forceinline__ f2 dtf11(float x0, float x1, float y0) {
    float q, r;
    div_rem(x0, y0, q, r);
    return {q, __fdiv_rn(__fadd_rn(r, x1), y0)};
}
__device__ __forceinline__ f2 dtf1(float x0, float x1, float y0, float y1) {
    float q, r0;
    div_rem(x0, y0, q, r0);
    const float r1 = __fmaf_rn(-q, y1, x1);
    return {q, __fdiv_rn(__fadd_rn(r0, r1), __fadd_rn(y0, y1))};
}
// DPF1 (coupled): divisor y0.
__device__ __forceinline__ f2 dpf1(float x0, float x1, float y0, float y1) {
    float q, r0;
    div_rem(x0, y0, q, r0);
    const float r1 = __fmaf_rn(-q, y1, x1);
    return {q, __fdiv_rn(__fadd_rn(r0, r1), y0)};
}
__device__ __forceinline__ f2 rpf1(float x0, float x1) {
    float c, d;
    sqrt_rem(x0, c, d);
    return {c, __fdiv_rn(__fadd_rn(x1, d), __fmul_rn(2.0f, c))};
}
__device__ __forceinline__ f2 rpf11(float x0) {
    float c, d;
    sqrt_rem(x0, c, d);
    return {c, __fdiv_rn(d, __fmul_rn(2.0f, c))};
}
// RTF1 (steps as in the binary64 version).
__device__ __forceinline__ f2 rtf1(float x0, float x1) {
    const float z0 = __fsqrt_rn(x0);
    float u0, u1;
    two_sum(x0, x1, u0, u1);
    const f2 v = rpf1(u0, u1);
    const f2 w = stf11(v.z0, v.z1, z0);
    return {z0, __fadd_rn(w.z0, w.z1)};
}

// Algorithm 1.1 (Fast Two-Sum), literal: renormalisation.
__device__ __forceinline__ f2 renorm(f2 z) {
    const float s = __fadd_rn(z.z0, z.z1);
    const float bv = __fsub_rn(s, z.z0);
    return {s, __fsub_rn(z.z1, bv)};
}

// Operand kinds (as the binary64 apply()).
__device__ __forceinline__ f2 apply(int op, float x0, float x1, bool xd, float y0, float y1, bool yd) {
    if (op == OP_SQRT) return xd ? rpf11(x0) : rtf1(x0, x1);
    if (xd && yd) {
        f2 z;
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
    if (xd) x1 = 0.0f;
    switch (op) {
    case OP_ADD: return atf1(x0, x1, y0, y1);
    case OP_SUB: return stf1(x0, x1, y0, y1);
    case OP_MUL: return mtf1(x0, x1, y0, y1);
    default: return dtf1(x0, x1, y0, y1);
    }
}

__device__ __forceinline__ f2 apply_coupled(int op, float x0, float x1, bool xd, float y0, float y1, bool yd) {
    const int base = op - 5;
    if (base == OP_SQRT) return xd ? rpf11(x0) : renorm(rpf1(x0, x1));
    if (xd && yd) return apply(base, x0, x1, true, y0, y1, true);
    if (yd) {
        switch (base) {
        case OP_ADD: return renorm(atf11(x0, x1, y0));
        case OP_SUB: return renorm(stf11(x0, x1, y0));
        case OP_MUL: return renorm(mtf11(x0, x1, y0));
        default: return renorm(dtf11(x0, x1, y0));
        }
    }
    if (xd) x1 = 0.0f;
    switch (base) {
    case OP_ADD: return renorm(atf1(x0, x1, y0, y1));
    case OP_SUB: return renorm(stf1(x0, x1, y0, y1));
    case OP_MUL: return renorm(mpf1(x0, x1, y0, y1));
    default: return renorm(dpf1(x0, x1, y0, y1));
    }
}

template <bool P>
__device__ __forceinline__ f2 apply_any(int op, float x0, float x1, bool xd, float y0, float y1, bool yd) {
    if (P && op > OP_SQRT) return apply_coupled(op, x0, x1, xd, y0, y1, yd);
    return apply(op, x0, x1, xd, y0, y1, yd);
}

__device__ __forceinline__ float apply_plain(int op, float a, float b) {
    if (op > OP_SQRT) op -= 5;
    switch (op) {
    case OP_ADD: return __fadd_rn(a, b);
    case OP_SUB: return __fsub_rn(a, b);
    case OP_MUL: return __fmul_rn(a, b);
    case OP_DIV: return __fdiv_rn(a, b);
    default: return __fsqrt_rn(a);
    }
}

// Panic flag of binary32 results: |z1| > tau (*) |z0| (REL) or
// |z1| > m (*) ulp(z0) (ULP), ulp(v) = 2^(max(e,-126)-23); mode bit 4 is the
// sticky flag (applied by the program kernels).
struct FlagCfg32 {
    int mode;
    float tau, m;
};

__device__ __forceinline__ float ulp_of(float v) {
    int e = (int)((__float_as_uint(v) >> 23) & 0xFF);
    if (e == 0xFF) return __uint_as_float(0x7FC00000u);
    if (e == 0) e = 1;
    const int p = e - 150;                      // exponent of the ulp, >= -149
    if (p >= -126) return __uint_as_float((uint32_t)(p + 127) << 23);
    return __uint_as_float(1u << (p + 149));
}

__device__ __forceinline__ uint8_t flag_of(float z0, float z1, const FlagCfg32 &f) {
    uint8_t r = 0;
    const uint32_t e0 = (__float_as_uint(z0) >> 23) & 0xFF, e1 = (__float_as_uint(z1) >> 23) & 0xFF;
    if (e0 == 0xFF || e1 == 0xFF) r |= 2;
    const float lim = (f.mode & 3) == 0 ? __fmul_rn(f.tau, fabsf(z0)) : __fmul_rn(f.m, ulp_of(z0));
    if (fabsf(z1) > lim) r |= 1;
    return r;
}

}  // namespace tf
