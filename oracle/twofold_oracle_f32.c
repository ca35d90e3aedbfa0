/*
 * CPU oracle, binary32 basis: the twofold algorithms of twofold_oracle.c
 * with float numbers (the paper's C++ types are generic over float and
 * double; its application logs print both).  TEST INFRASTRUCTURE ONLY, like
 * twofold_oracle.c, and sharing no code with the CUDA library.
 *
 * Every operation is a binary32 operation, one per statement, round to
 * nearest even, compiled with -ffp-contract=off; fmaf() is the correctly
 * rounded fused multiply-add and sqrtf() the correctly rounded root.  The
 * readings R1-R10 of twofold_oracle.c apply unchanged.  Two more:
 *  R11 Panic flag of binary32 results: the same rule with float arithmetic
 *      (|z1| > tau (*) |z0| or |z1| > m ulp(z0), ulp(v) = 2^(max(e,-126)-23));
 *      the threshold is the caller's (a default is the interface's choice).
 *  R12 Sticky flag (mode bit 4, both bases): the flag of a program's result
 *      ORs the flags of every instruction's result, so a loss anywhere in a
 *      chain stays visible at its end.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

typedef struct { float z0, z1; } tfof_tf;

/* =========================================================== Background */

/* Algorithm 1.2 (Two-Sum). */
void tfof_two_sum(float a, float b, float *s, float *t) {
    float s_ = a + b;
    float b1 = s_ - a;
    float a1 = s_ - b1;
    float bs = b - b1;
    float as = a - a1;
    *s = s_;
    *t = as + bs;
}

/* Algorithm 2.2 (Two-Diff), R1: b# = b' - b, a# = a - a'. */
void tfof_two_diff(float a, float b, float *d, float *t) {
    float d_ = a - b;
    float b1 = a - d_;
    float a1 = b1 + d_;
    float bs = b1 - b;
    float as = a - a1;
    *d = d_;
    *t = as + bs;
}

/* Algorithm 1.1 (Fast Two-Sum), three operations (R10). */
void tfof_fast_two_sum(float a, float b, float *s, float *t) {
    float s_ = a + b;
    float b1 = s_ - a;
    *s = s_;
    *t = b - b1;
}

/* Algorithm 3 (Two-Product with FMA). */
void tfof_two_prod(float a, float b, float *p, float *e) {
    float p_ = a * b;
    *p = p_;
    *e = fmaf(a, b, -p_);
}

/* Algorithm 4: q = a/b, r = fma(-q, b, a) (R3). */
void tfof_div_rem(float a, float b, float *q, float *r) {
    float q_ = a / b;
    *q = q_;
    *r = fmaf(-q_, b, a);
}

/* Algorithm 5: c = sqrt(a), d = fma(-c, c, a) (R3). */
void tfof_sqrt_rem(float a, float *c, float *d) {
    float c_ = sqrtf(a);
    *c = c_;
    *d = fmaf(-c_, c_, a);
}

/* =========================================================== Algorithms */

tfof_tf tfof_atf1(float x0, float x1, float y0, float y1) {
    tfof_tf z;
    float s, e;
    tfof_two_sum(x0, y0, &s, &e);
    float u = x1 + y1;
    z.z0 = s;
    z.z1 = u + e;
    return z;
}

tfof_tf tfof_atf11(float x0, float x1, float y0) {
    tfof_tf z;
    float s, e;
    tfof_two_sum(x0, y0, &s, &e);
    z.z0 = s;
    z.z1 = x1 + e;
    return z;
}

tfof_tf tfof_stf1(float x0, float x1, float y0, float y1) {
    tfof_tf z;
    float d, e;
    tfof_two_diff(x0, y0, &d, &e);
    float u = x1 - y1;
    z.z0 = d;
    z.z1 = u + e;
    return z;
}

tfof_tf tfof_stf11(float x0, float x1, float y0) {
    tfof_tf z;
    float d, e;
    tfof_two_diff(x0, y0, &d, &e);
    z.z0 = d;
    z.z1 = x1 + e;
    return z;
}

/* MTF1: z1 = e00 (+) p11 (+) (p01 (+) p10). */
tfof_tf tfof_mtf1(float x0, float x1, float y0, float y1) {
    tfof_tf z;
    float p00, e00;
    tfof_two_prod(x0, y0, &p00, &e00);
    float p11 = x1 * y1;
    float p01 = x0 * y1;
    float p10 = x1 * y0;
    float u = e00 + p11;
    float v = p01 + p10;
    z.z0 = p00;
    z.z1 = u + v;
    return z;
}

tfof_tf tfof_mtf11(float x0, float x1, float y0) {
    tfof_tf z;
    float p00, e00;
    tfof_two_prod(x0, y0, &p00, &e00);
    float p10 = x1 * y0;
    z.z0 = p00;
    z.z1 = e00 + p10;
    return z;
}

/* MPF1 (coupled): z1 = e00 (+) (p01 (+) p10). */
tfof_tf tfof_mpf1(float x0, float x1, float y0, float y1) {
    tfof_tf z;
    float p00, e00;
    tfof_two_prod(x0, y0, &p00, &e00);
    float p01 = x0 * y1;
    float p10 = x1 * y0;
    float v = p01 + p10;
    z.z0 = p00;
    z.z1 = e00 + v;
    return z;
}

tfof_tf tfof_dtf111(float x0, float y0) {
    tfof_tf z;
    float q, r1;
    tfof_div_rem(x0, y0, &q, &r1);
    z.z0 = q;
    z.z1 = r1 / y0;
    return z;
}

tfof_tf tfof_dtf11(float x0, float x1, float y0) {
    tfof_tf z;
    float q, r;
    tfof_div_rem(x0, y0, &q, &r);
    float c = r + x1;
    z.z0 = q;
    z.z1 = c / y0;
    return z;
}

tfof_tf tfof_dtf1(float x0, float x1, float y0, float y1) {
    tfof_tf z;
    float q, r0;
    tfof_div_rem(x0, y0, &q, &r0);
    float r1 = fmaf(-q, y1, x1);
    float c0 = r0 + r1;
    float d0 = y0 + y1;
    z.z0 = q;
    z.z1 = c0 / d0;
    return z;
}

/* DPF1 (coupled): divisor y0. */
tfof_tf tfof_dpf1(float x0, float x1, float y0, float y1) {
    tfof_tf z;
    float q, r0;
    tfof_div_rem(x0, y0, &q, &r0);
    float r1 = fmaf(-q, y1, x1);
    float c0 = r0 + r1;
    z.z0 = q;
    z.z1 = c0 / y0;
    return z;
}

tfof_tf tfof_rpf1(float x0, float x1) {
    tfof_tf z;
    float c, d;
    tfof_sqrt_rem(x0, &c, &d);
    float t = x1 + d;
    float w = 2.0f * c;
    z.z0 = c;
    z.z1 = t / w;
    return z;
}

tfof_tf tfof_rpf11(float x0) {
    tfof_tf z;
    float c, d;
    tfof_sqrt_rem(x0, &c, &d);
    float w = 2.0f * c;
    z.z0 = c;
    z.z1 = d / w;
    return z;
}

/* RTF1 (R5). */
tfof_tf tfof_rtf1(float x0, float x1) {
    tfof_tf z;
    float z0 = sqrtf(x0);
    float u0, u1;
    tfof_two_sum(x0, x1, &u0, &u1);
    tfof_tf v = tfof_rpf1(u0, u1);
    tfof_tf w = tfof_stf11(v.z0, v.z1, z0);
    z.z0 = z0;
    z.z1 = w.z0 + w.z1;
    return z;
}

/* ------------------------------------------- operand kinds (R6, R10) */
enum { F_ADD = 1, F_SUB = 2, F_MUL = 3, F_DIV = 4, F_SQRT = 5, F_PADD = 6, F_PSQRT = 10 };

static tfof_tf kinds(int op, float x0, float x1, int xd, float y0, float y1, int yd) {
    tfof_tf z;
    if (op == F_SQRT) return xd ? tfof_rpf11(x0) : tfof_rtf1(x0, x1);
    if (xd && yd) {
        switch (op) {
        case F_ADD: tfof_two_sum(x0, y0, &z.z0, &z.z1); return z;
        case F_SUB: tfof_two_diff(x0, y0, &z.z0, &z.z1); return z;
        case F_MUL: tfof_two_prod(x0, y0, &z.z0, &z.z1); return z;
        default:    return tfof_dtf111(x0, y0);
        }
    }
    if (yd) {
        switch (op) {
        case F_ADD: return tfof_atf11(x0, x1, y0);
        case F_SUB: return tfof_stf11(x0, x1, y0);
        case F_MUL: return tfof_mtf11(x0, x1, y0);
        default:    return tfof_dtf11(x0, x1, y0);
        }
    }
    if (xd) x1 = 0.0f;
    switch (op) {
    case F_ADD: return tfof_atf1(x0, x1, y0, y1);
    case F_SUB: return tfof_stf1(x0, x1, y0, y1);
    case F_MUL: return tfof_mtf1(x0, x1, y0, y1);
    default:    return tfof_dtf1(x0, x1, y0, y1);
    }
}

static tfof_tf renorm(tfof_tf z) {
    tfof_tf r;
    tfof_fast_two_sum(z.z0, z.z1, &r.z0, &r.z1);
    return r;
}

static tfof_tf coupled(int op, float x0, float x1, int xd, float y0, float y1, int yd) {
    int base = op - 5;
    if (base == F_SQRT) return xd ? tfof_rpf11(x0) : renorm(tfof_rpf1(x0, x1));
    if (xd && yd) return kinds(base, x0, x1, 1, y0, y1, 1);
    if (yd) {
        switch (base) {
        case F_ADD: return renorm(tfof_atf11(x0, x1, y0));
        case F_SUB: return renorm(tfof_stf11(x0, x1, y0));
        case F_MUL: return renorm(tfof_mtf11(x0, x1, y0));
        default:    return renorm(tfof_dtf11(x0, x1, y0));
        }
    }
    if (xd) x1 = 0.0f;
    switch (base) {
    case F_ADD: return renorm(tfof_atf1(x0, x1, y0, y1));
    case F_SUB: return renorm(tfof_stf1(x0, x1, y0, y1));
    case F_MUL: return renorm(tfof_mpf1(x0, x1, y0, y1));
    default:    return renorm(tfof_dpf1(x0, x1, y0, y1));
    }
}

static tfof_tf any(int op, float x0, float x1, int xd, float y0, float y1, int yd) {
    return op >= F_PADD ? coupled(op, x0, x1, xd, y0, y1, yd) : kinds(op, x0, x1, xd, y0, y1, yd);
}

void tfof_op(int op, float x0, float x1, int xd, float y0, float y1, int yd, float *z0, float *z1) {
    tfof_tf z = any(op, x0, x1, xd, y0, y1, yd);
    *z0 = z.z0;
    *z1 = z.z1;
}

/* ----------------------------------------------------------- panic flag (R11) */
static float ulpf_of(float v) {
    uint32_t b;
    memcpy(&b, &v, 4);
    int e = (int)((b >> 23) & 0xFF);
    if (e == 0) e = 1;
    if (e == 0xFF) return NAN;
    return ldexpf(1.0f, e - 150);
}

unsigned char tfof_flag(float z0, float z1, int mode, float tau, float m) {
    unsigned char f = 0;
    if (!isfinite(z0) || !isfinite(z1)) f |= 2;
    float lim = ((mode & 3) == 0) ? tau * fabsf(z0) : m * ulpf_of(z0);
    if (fabsf(z1) > lim) f |= 1;
    return f;
}

/* ------------------------------------------------------- elementwise programs */
#define TFOF_MAXREG 32

void tfof_ew(const int32_t *prog, int nprog, const float *const *in_hi, const float *const *in_lo, int nin,
             int64_t i0, int64_t i1, float *out_hi, float *out_lo, unsigned char *flags, int mode, float tau,
             float m) {
    for (int64_t i = i0; i < i1; ++i) {
        float r0[TFOF_MAXREG], r1[TFOF_MAXREG];
        int dotted[TFOF_MAXREG];
        for (int k = 0; k < nin; ++k) {
            r0[k] = in_hi[k][i];
            r1[k] = in_lo[k] ? in_lo[k][i] : 0.0f;
            dotted[k] = in_lo[k] == NULL;
        }
        int dst = 0;
        unsigned char sticky = 0;
        for (int s = 0; s < nprog; ++s) {
            int op = prog[4 * s], a = prog[4 * s + 2], b = prog[4 * s + 3];
            dst = prog[4 * s + 1];
            if (op == F_SQRT || op == F_PSQRT) b = a;
            tfof_tf z = any(op, r0[a], r1[a], dotted[a], r0[b], r1[b], dotted[b]);
            r0[dst] = z.z0;
            r1[dst] = z.z1;
            dotted[dst] = 0;
            if (mode & 4) sticky |= tfof_flag(z.z0, z.z1, mode, tau, m);
        }
        out_hi[i] = r0[dst];
        out_lo[i] = r1[dst];
        if (flags) flags[i] = (unsigned char)(tfof_flag(r0[dst], r1[dst], mode, tau, m) | sticky);
    }
}

void tfof_ew_plain(const int32_t *prog, int nprog, const float *const *in_hi, int nin, int64_t i0, int64_t i1,
                   float *out) {
    for (int64_t i = i0; i < i1; ++i) {
        float r[TFOF_MAXREG];
        for (int k = 0; k < nin; ++k) r[k] = in_hi[k][i];
        int dst = 0;
        for (int s = 0; s < nprog; ++s) {
            int op = prog[4 * s], a = prog[4 * s + 2], b = prog[4 * s + 3];
            dst = prog[4 * s + 1];
            if (op >= F_PADD) op -= 5;
            if (op == F_SQRT) b = a;
            float v;
            switch (op) {
            case F_ADD: v = r[a] + r[b]; break;
            case F_SUB: v = r[a] - r[b]; break;
            case F_MUL: v = r[a] * r[b]; break;
            case F_DIV: v = r[a] / r[b]; break;
            default:    v = sqrtf(r[a]); break;
            }
            r[dst] = v;
        }
        out[i] = r[dst];
    }
}

/* ----------------------------------------------- sum and dot in the order R8
 * (binary32): leaves of L elements from (+0, +0); a sum adds each element
 * with ATF1 (ATF1.1 when the input is dotted), a dot adds each product
 * x_i * y_i, formed as a twofold by the multiplication of the operand kinds
 * (Two-Product for two dotted operands, MTF1.1 / MTF1 otherwise), with
 * ATF1; then the pairwise tree of ATF1 with the odd node carried. */
void tfof_reduce(const float *xh, const float *xl, const float *yh, const float *yl, int64_t n, int64_t L,
                 int is_dot, float *z0, float *z1) {
    int64_t m = n ? (n + L - 1) / L : 0;
    if (m == 0) { *z0 = 0.0f; *z1 = 0.0f; return; }
    tfof_tf *nodes = (tfof_tf *)malloc(sizeof(tfof_tf) * (size_t)m);
    for (int64_t j = 0; j < m; ++j) {
        tfof_tf acc = {0.0f, 0.0f};
        int64_t e = (j + 1) * L < n ? (j + 1) * L : n;
        for (int64_t i = j * L; i < e; ++i) {
            if (!is_dot) {
                acc = xl ? tfof_atf1(acc.z0, acc.z1, xh[i], xl[i]) : tfof_atf11(acc.z0, acc.z1, xh[i]);
            } else {
                tfof_tf q = kinds(F_MUL, xh[i], xl ? xl[i] : 0.0f, xl == NULL, yh[i], yl ? yl[i] : 0.0f, yl == NULL);
                acc = tfof_atf1(acc.z0, acc.z1, q.z0, q.z1);
            }
        }
        nodes[j] = acc;
    }
    while (m > 1) {
        int64_t h = 0;
        for (int64_t i = 0; i + 1 < m; i += 2) nodes[h++] = tfof_atf1(nodes[i].z0, nodes[i].z1, nodes[i + 1].z0, nodes[i + 1].z1);
        if (m & 1) nodes[h++] = nodes[m - 1];
        m = h;
    }
    *z0 = nodes[0].z0;
    *z1 = nodes[0].z1;
    free(nodes);
}

void tfof_reduce_sum(const float *xh, const float *xl, int64_t n, int64_t L, float *z0, float *z1) {
    tfof_reduce(xh, xl, NULL, NULL, n, L, 0, z0, z1);
}

/* Plain binary32 twin: the same leaves and tree with s = +0 and
 * s = s + x_i (sum) or s = s + x_i * y_i (separate multiply and add). */
float tfof_reduce_plain(const float *x, const float *y, int64_t n, int64_t L, int is_dot) {
    int64_t m = n ? (n + L - 1) / L : 0;
    if (m == 0) return 0.0f;
    float *nodes = (float *)malloc(sizeof(float) * (size_t)m);
    for (int64_t j = 0; j < m; ++j) {
        float s = 0.0f;
        int64_t e = (j + 1) * L < n ? (j + 1) * L : n;
        for (int64_t i = j * L; i < e; ++i) {
            if (is_dot) { float q = x[i] * y[i]; s = s + q; }
            else        s = s + x[i];
        }
        nodes[j] = s;
    }
    while (m > 1) {
        int64_t h = 0;
        for (int64_t i = 0; i + 1 < m; i += 2) nodes[h++] = nodes[i] + nodes[i + 1];
        if (m & 1) nodes[h++] = nodes[m - 1];
        m = h;
    }
    float r = nodes[0];
    free(nodes);
    return r;
}
