/*
 * CPU oracle for twofold fast arithmetic (Latkin, "Twofold fast arithmetic",
 * arXiv:1401.6235).  TEST INFRASTRUCTURE ONLY: the tests, the package smoke
 * check and the CPU-baseline leg of the benchmark call it; the library's
 * product path never does.  It shares no code with the CUDA library.
 *
 * Plain, slow, obviously correct: every twofold algorithm is written out in
 * the paper's order and notation, one IEEE binary64 operation per statement,
 * round-to-nearest-even, compiled with -ffp-contract=off so that no a*b+c is
 * fused behind our back.  fma() is the C99 correctly rounded fused
 * multiply-add, sqrt() the correctly rounded square root.
 *
 * Notation: x = x0 + x1, y = y0 + y1 are twofolds; a "dotted" operand is a
 * plain double (tail absent).  Sums of three terms associate to the left
 * (Background, "Dekker arithmetic").
 *
 * Readings of the paper taken here (the paper is silent, garbled or
 * inconsistent at these points):
 *  R1  Algorithm 2.2 (Two-Diff) as printed gives -t: steps (4),(5) are read
 *      as b# = b' - b, a# = a - a' (Shewchuk's order), so a - b = d + t.
 *  R2  err(a+b) / err(a-b) are Algorithm 1.2 / 2.2 (the general forms; the
 *      operands of a twofold op are not ordered by magnitude).
 *  R3  The remainder of Algorithm 4 is fma(-q, b, a) (Fragment 4); the
 *      sqrt residual of Algorithm 5 is fma(-c, c, a).
 *  R4  "/2z0" in RPF 1 / RPF 1.1 is division by (2*z0).
 *  R5  RTF 1 step (2) renormalises with Two-Sum (Algorithm 1.2), step (3) is
 *      RPF 1 on (u0, u1), step (4) is STF 1.1 of (v0, v1) and z0.
 *  R6  Operand kinds: (twofold, twofold) -> general algorithm; (twofold,
 *      dotted) -> the ".1" algorithm; (dotted, twofold) -> general algorithm
 *      with x1 = +0; (dotted, dotted) -> the exact transform (Two-Sum,
 *      Two-Diff, Two-Product) or DTF 1.1.1; sqrt of a dotted value -> RPF 1.1.
 *  R7  No special cases (Algorithms, "Methodic"): NaN/Inf flow through the
 *      basic operations; e.g. sqrt(+0) gives z1 = 0/0 = NaN.
 *  R8  Sum and dot order (the paper fixes none): consecutive leaves of L
 *      elements, each summed left to right from (+0, +0) into a twofold
 *      accumulator; then a bottom-up pairwise tree over the leaf results,
 *      node i of level j+1 = ATF1(node 2i, node 2i+1), an odd last node is
 *      carried up unchanged.
 *  R9  Panic flag (idea: Motivation, Applications; threshold not in the
 *      paper): bit0 PANIC if |z1| > tau*|z0| (REL) or |z1| > m*ulp(z0) (ULP);
 *      bit1 NONFINITE if z0 or z1 is NaN or infinite.
 *  R10 "Coupled" (Dekker emulation) operations, the paper's p-prefixed
 *      functions: add/subtract use ATF/STF (no special coupled algorithm
 *      exists), multiply MPF 1 (MTF 1.1 when y is dotted), divide DPF 1
 *      (DTF 1.1 when y is dotted), root RPF 1; the output is then
 *      renormalised with Fast Two-Sum (Algorithm 1.1, its three operations
 *      taken literally; Dekker arithmetic section, Applications).  With every
 *      operand dotted the output of the exact transform / DTF 1.1.1 / RPF 1.1
 *      is already coupled and is returned as is (Applications; the pdiv of
 *      two dotted numbers in Fragment 4 returns tdiv unchanged).
 *  R12 Sticky flag (mode bit 4): a program's flag ORs the flags of every
 *      instruction's result (twofold_oracle_f32.c holds the binary32 basis).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>

/* ---------------------------------------------------------------- types */
typedef struct { double z0, z1; } tfo_tf;

/* =========================================================== Background */

/* Algorithm 1.2 (Two-Sum): a + b -> s + t for arbitrary a, b. */
void tfo_two_sum(double a, double b, double *s, double *t) {
    double s_ = a + b;          /* (1) s  = a (+) b   */
    double b1 = s_ - a;         /* (2) b' = s (-) a   */
    double a1 = s_ - b1;        /* (3) a' = s (-) b'  */
    double bs = b - b1;         /* (4) b# = b (-) b'  */
    double as = a - a1;         /* (5) a# = a (-) a'  */
    *s = s_;
    *t = as + bs;               /* (6) t  = a# (+) b# */
}

/* Algorithm 2.2 (Two-Diff): a - b -> d + t for arbitrary a, b, with the
 * signs of steps (4),(5) read as in Shewchuk (reading R1). */
void tfo_two_diff(double a, double b, double *d, double *t) {
    double d_ = a - b;          /* (1) d  = a (-) b   */
    double b1 = a - d_;         /* (2) b' = a (-) d   */
    double a1 = b1 + d_;        /* (3) a' = b' (+) d  */
    double bs = b1 - b;         /* (4) b# = b' (-) b  */
    double as = a - a1;         /* (5) a# = a (-) a'  */
    *d = d_;
    *t = as + bs;               /* (6) t  = a# (+) b# */
}

/* Algorithm 3 (Two-Product-FMA): a * b -> p + e, e = fl(ab - p). */
void tfo_two_prod(double a, double b, double *p, double *e) {
    double p_ = a * b;
    *p = p_;
    *e = fma(a, b, -p_);
}

/* Algorithm 4: a / b -> q, r with r = fl(a - qb) = fma(-q, b, a) (R3). */
void tfo_div_rem(double a, double b, double *q, double *r) {
    double q_ = a / b;
    *q = q_;
    *r = fma(-q_, b, a);
}

/* Algorithm 5: sqrt(a) -> c, d with d = fl(a - c^2) = fma(-c, c, a) (R3). */
void tfo_sqrt_rem(double a, double *c, double *d) {
    double c_ = sqrt(a);
    *c = c_;
    *d = fma(-c_, c_, a);
}

/* Algorithm 1.1 (Fast Two-Sum): a + b -> s + t, exact when |a| >= |b|.
 * Used to renormalise a twofold (Dekker arithmetic section), three
 * operations taken literally whatever the magnitudes. */
void tfo_fast_two_sum(double a, double b, double *s, double *t) {
    double s_ = a + b;          /* (1) s  = a (+) b   */
    double b1 = s_ - a;         /* (2) b' = s (-) a   */
    *s = s_;
    *t = b - b1;                /* (3) t  = b (-) b'  */
}

/* =========================================================== Algorithms */

/* ATF1: z0 = x0 (+) y0;  z1 = x1 (+) y1 (+) err(x0 + y0). */
tfo_tf tfo_atf1(double x0, double x1, double y0, double y1) {
    tfo_tf z;
    double s, e;
    tfo_two_sum(x0, y0, &s, &e);
    z.z0 = s;
    double u = x1 + y1;
    z.z1 = u + e;
    return z;
}

/* ATF1.1 (y1 = 0): z0 = x0 (+) y0;  z1 = x1 (+) err(x0 + y0). */
tfo_tf tfo_atf11(double x0, double x1, double y0) {
    tfo_tf z;
    double s, e;
    tfo_two_sum(x0, y0, &s, &e);
    z.z0 = s;
    z.z1 = x1 + e;
    return z;
}

/* STF1: z0 = x0 (-) y0;  z1 = x1 (-) y1 (+) err(x0 - y0). */
tfo_tf tfo_stf1(double x0, double x1, double y0, double y1) {
    tfo_tf z;
    double d, e;
    tfo_two_diff(x0, y0, &d, &e);
    z.z0 = d;
    double u = x1 - y1;
    z.z1 = u + e;
    return z;
}

/* STF1.1 (y1 = 0): z0 = x0 (-) y0;  z1 = x1 (+) err(x0 - y0). */
tfo_tf tfo_stf11(double x0, double x1, double y0) {
    tfo_tf z;
    double d, e;
    tfo_two_diff(x0, y0, &d, &e);
    z.z0 = d;
    z.z1 = x1 + e;
    return z;
}

/* MTF1: x_i * y_j -> p_ij + e_ij (only e00 is needed);
 *       z0 = p00;  z1 = e00 (+) p11 (+) (p01 (+) p10). */
tfo_tf tfo_mtf1(double x0, double x1, double y0, double y1) {
    tfo_tf z;
    double p00, e00;
    tfo_two_prod(x0, y0, &p00, &e00);
    double p11 = x1 * y1;
    double p01 = x0 * y1;
    double p10 = x1 * y0;
    double u = e00 + p11;
    double v = p01 + p10;
    z.z0 = p00;
    z.z1 = u + v;
    return z;
}

/* MTF1.1 (y1 = 0): z0 = p00;  z1 = e00 (+) p10. */
tfo_tf tfo_mtf11(double x0, double x1, double y0) {
    tfo_tf z;
    double p00, e00;
    tfo_two_prod(x0, y0, &p00, &e00);
    double p10 = x1 * y0;
    z.z0 = p00;
    z.z1 = e00 + p10;
    return z;
}

/* DTF1.1.1 (x1 = y1 = 0): z0 = fl(x0/y0); r1 = fma(x0 - z0 y0); z1 = fl(r1/y0). */
tfo_tf tfo_dtf111(double x0, double y0) {
    tfo_tf z;
    double q, r1;
    tfo_div_rem(x0, y0, &q, &r1);
    z.z0 = q;
    z.z1 = r1 / y0;
    return z;
}

/* DTF1.1 (y1 = 0): z0 = fl(x0/y0); r = fma(x0 - z0 y0); c = r (+) x1; z1 = fl(c/y0). */
tfo_tf tfo_dtf11(double x0, double x1, double y0) {
    tfo_tf z;
    double q, r;
    tfo_div_rem(x0, y0, &q, &r);
    double c = r + x1;
    z.z0 = q;
    z.z1 = c / y0;
    return z;
}

/* DTF1: z0 = fl(x0/y0); r0 = fma(x0 - z0 y0); r1 = fma(x1 - z0 y1);
 *       c0 = r0 (+) r1; d0 = y0 (+) y1; z1 = fl(c0/d0). */
tfo_tf tfo_dtf1(double x0, double x1, double y0, double y1) {
    tfo_tf z;
    double q, r0;
    tfo_div_rem(x0, y0, &q, &r0);
    double r1 = fma(-q, y1, x1);
    double c0 = r0 + r1;
    double d0 = y0 + y1;
    z.z0 = q;
    z.z1 = c0 / d0;
    return z;
}

/* MPF1 (coupled x, y): x_i * y_j -> p_ij + e_ij; z0 = p00;
 *       z1 = e00 (+) (p01 (+) p10)   (p11 omitted: minor for coupled input). */
tfo_tf tfo_mpf1(double x0, double x1, double y0, double y1) {
    tfo_tf z;
    double p00, e00;
    tfo_two_prod(x0, y0, &p00, &e00);
    double p01 = x0 * y1;
    double p10 = x1 * y0;
    double v = p01 + p10;
    z.z0 = p00;
    z.z1 = e00 + v;
    return z;
}

/* DPF1 (coupled x, y): z0 = fl(x0/y0); r0 = fma(x0 - z0 y0); r1 = fma(x1 - z0 y1);
 *       c0 = r0 (+) r1; z1 = fl(c0/y0)   (y0 + y1 is not renormalised). */
tfo_tf tfo_dpf1(double x0, double x1, double y0, double y1) {
    tfo_tf z;
    double q, r0;
    tfo_div_rem(x0, y0, &q, &r0);
    double r1 = fma(-q, y1, x1);
    double c0 = r0 + r1;
    z.z0 = q;
    z.z1 = c0 / y0;
    return z;
}

/* RPF1 (coupled input): z0 = sqrt(x0); z1 = (x1 (+) fma(x0 - z0^2)) / (2 z0). */
tfo_tf tfo_rpf1(double x0, double x1) {
    tfo_tf z;
    double c, d;
    tfo_sqrt_rem(x0, &c, &d);
    double t = x1 + d;
    double w = 2.0 * c;
    z.z0 = c;
    z.z1 = t / w;
    return z;
}

/* RPF1.1 (x1 = 0): z0 = sqrt(x0); z1 = fma(x0 - z0^2) / (2 z0). */
tfo_tf tfo_rpf11(double x0) {
    tfo_tf z;
    double c, d;
    tfo_sqrt_rem(x0, &c, &d);
    double w = 2.0 * c;
    z.z0 = c;
    z.z1 = d / w;
    return z;
}

/* RTF1: (1) z0 = sqrt(x0); (2) x0 + x1 -> u0 + u1 (Two-Sum);
 *       (3) RPF1(u0, u1) -> v0 + v1; (4) STF1.1: (v0 + v1) (-) z0 -> w0 + w1;
 *       (5) z1 = w0 (+) w1. */
tfo_tf tfo_rtf1(double x0, double x1) {
    tfo_tf z;
    double z0 = sqrt(x0);
    double u0, u1;
    tfo_two_sum(x0, x1, &u0, &u1);
    tfo_tf v = tfo_rpf1(u0, u1);
    tfo_tf w = tfo_stf11(v.z0, v.z1, z0);
    z.z0 = z0;
    z.z1 = w.z0 + w.z1;
    return z;
}

/* ------------------------------------------- operand-kind dispatch (R6) */
enum { TFO_ADD = 1, TFO_SUB = 2, TFO_MUL = 3, TFO_DIV = 4, TFO_SQRT = 5 };

static tfo_tf op_kinds(int op, double x0, double x1, int xd, double y0, double y1, int yd) {
    tfo_tf z;
    if (op == TFO_SQRT) return xd ? tfo_rpf11(x0) : tfo_rtf1(x0, x1);
    if (xd && yd) {
        switch (op) {
        case TFO_ADD: tfo_two_sum(x0, y0, &z.z0, &z.z1); return z;
        case TFO_SUB: tfo_two_diff(x0, y0, &z.z0, &z.z1); return z;
        case TFO_MUL: tfo_two_prod(x0, y0, &z.z0, &z.z1); return z;
        default:      return tfo_dtf111(x0, y0);
        }
    }
    if (yd) {
        switch (op) {
        case TFO_ADD: return tfo_atf11(x0, x1, y0);
        case TFO_SUB: return tfo_stf11(x0, x1, y0);
        case TFO_MUL: return tfo_mtf11(x0, x1, y0);
        default:      return tfo_dtf11(x0, x1, y0);
        }
    }
    if (xd) x1 = 0.0;
    switch (op) {
    case TFO_ADD: return tfo_atf1(x0, x1, y0, y1);
    case TFO_SUB: return tfo_stf1(x0, x1, y0, y1);
    case TFO_MUL: return tfo_mtf1(x0, x1, y0, y1);
    default:      return tfo_dtf1(x0, x1, y0, y1);
    }
}

/* Renormalise z0 + z1 with Fast Two-Sum (R10). */
static tfo_tf renorm(tfo_tf z) {
    tfo_tf r;
    tfo_fast_two_sum(z.z0, z.z1, &r.z0, &r.z1);
    return r;
}

/* Coupled ("p") operations, R10: op = TFO_PADD .. TFO_PSQRT. */
enum { TFO_PADD = 6, TFO_PSUB = 7, TFO_PMUL = 8, TFO_PDIV = 9, TFO_PSQRT = 10 };

static tfo_tf op_coupled(int op, double x0, double x1, int xd, double y0, double y1, int yd) {
    int base = op - 5;
    if (base == TFO_SQRT) return xd ? tfo_rpf11(x0) : renorm(tfo_rpf1(x0, x1));
    if (xd && yd) return op_kinds(base, x0, x1, 1, y0, y1, 1);     /* already coupled */
    if (yd) {
        switch (base) {
        case TFO_ADD: return renorm(tfo_atf11(x0, x1, y0));
        case TFO_SUB: return renorm(tfo_stf11(x0, x1, y0));
        case TFO_MUL: return renorm(tfo_mtf11(x0, x1, y0));     /* MPF1.1 = MTF1.1 */
        default:      return renorm(tfo_dtf11(x0, x1, y0));     /* DPF1.1 = DTF1.1 */
        }
    }
    if (xd) x1 = 0.0;
    switch (base) {
    case TFO_ADD: return renorm(tfo_atf1(x0, x1, y0, y1));
    case TFO_SUB: return renorm(tfo_stf1(x0, x1, y0, y1));
    case TFO_MUL: return renorm(tfo_mpf1(x0, x1, y0, y1));
    default:      return renorm(tfo_dpf1(x0, x1, y0, y1));
    }
}

static tfo_tf op_any(int op, double x0, double x1, int xd, double y0, double y1, int yd) {
    return op >= TFO_PADD ? op_coupled(op, x0, x1, xd, y0, y1, yd) : op_kinds(op, x0, x1, xd, y0, y1, yd);
}

/* Scalar entry for tests: kinds xd/yd = 1 means dotted. */
void tfo_op(int op, double x0, double x1, int xd, double y0, double y1, int yd,
            double *z0, double *z1) {
    tfo_tf z = op_any(op, x0, x1, xd, y0, y1, yd);
    *z0 = z.z0;
    *z1 = z.z1;
}

/* ----------------------------------------------------------- panic flag (R9) */
enum { TFO_PANIC = 1, TFO_NONFINITE = 2 };

static double ulp_of(double v) {
    uint64_t b;
    memcpy(&b, &v, 8);
    int e = (int)((b >> 52) & 0x7FF);
    if (e == 0) e = 1;
    if (e == 0x7FF) return NAN;
    return ldexp(1.0, e - 1075);
}

/* mode & 3: 0 = REL (|z1| > tau*|z0|), 1 = ULP (|z1| > m*ulp(z0)); mode & 4:
 * sticky (R12, applied by the program evaluator). */
unsigned char tfo_flag(double z0, double z1, int mode, double tau, double m) {
    unsigned char f = 0;
    if (!isfinite(z0) || !isfinite(z1)) f |= TFO_NONFINITE;
    double lim = ((mode & 3) == 0) ? tau * fabs(z0) : m * ulp_of(z0);
    if (fabs(z1) > lim) f |= TFO_PANIC;
    return f;
}

/* ------------------------------------------------------- elementwise programs
 * A program is a list of instructions {op, dst, a, b} over registers;
 * registers 0..nin-1 hold the inputs, the rest are temporaries.  Every
 * temporary is a general twofold; input i is dotted when its tail pointer is
 * NULL.  The result is the destination of the last instruction. */
#define TFO_MAXREG 32

void tfo_ew(const int32_t *prog, int nprog, const double *const *in_hi,
            const double *const *in_lo, int nin, int64_t i0, int64_t i1,
            double *out_hi, double *out_lo, unsigned char *flags,
            int mode, double tau, double m) {
    for (int64_t i = i0; i < i1; ++i) {
        double r0[TFO_MAXREG], r1[TFO_MAXREG];
        int dotted[TFO_MAXREG];
        for (int k = 0; k < nin; ++k) {
            r0[k] = in_hi[k][i];
            r1[k] = in_lo[k] ? in_lo[k][i] : 0.0;
            dotted[k] = in_lo[k] == NULL;
        }
        int dst = 0;
        unsigned char sticky = 0;
        for (int s = 0; s < nprog; ++s) {
            int op = prog[4 * s], a = prog[4 * s + 2], b = prog[4 * s + 3];
            dst = prog[4 * s + 1];
            if (op == TFO_SQRT || op == TFO_PSQRT) b = a;   /* unary: the second operand is unused */
            tfo_tf z = op_any(op, r0[a], r1[a], dotted[a], r0[b], r1[b], dotted[b]);
            r0[dst] = z.z0;
            r1[dst] = z.z1;
            dotted[dst] = 0;
            if (mode & 4) sticky |= tfo_flag(z.z0, z.z1, mode, tau, m);   /* R12 */
        }
        out_hi[i] = r0[dst];
        out_lo[i] = r1[dst];
        if (flags) flags[i] = (unsigned char)(tfo_flag(r0[dst], r1[dst], mode, tau, m) | sticky);
    }
}

/* Plain binary64 twin of a program: the same instructions on heads only. */
void tfo_ew_plain(const int32_t *prog, int nprog, const double *const *in_hi, int nin,
                  int64_t i0, int64_t i1, double *out) {
    for (int64_t i = i0; i < i1; ++i) {
        double r[TFO_MAXREG];
        for (int k = 0; k < nin; ++k) r[k] = in_hi[k][i];
        int dst = 0;
        for (int s = 0; s < nprog; ++s) {
            int op = prog[4 * s], a = prog[4 * s + 2], b = prog[4 * s + 3];
            dst = prog[4 * s + 1];
            if (op >= TFO_PADD) op -= 5;    /* the plain twin of a coupled op is the basic op */
            if (op == TFO_SQRT) b = a;
            double v;
            switch (op) {
            case TFO_ADD: v = r[a] + r[b]; break;
            case TFO_SUB: v = r[a] - r[b]; break;
            case TFO_MUL: v = r[a] * r[b]; break;
            case TFO_DIV: v = r[a] / r[b]; break;
            default:      v = sqrt(r[a]); break;
            }
            r[dst] = v;
        }
        out[i] = r[dst];
    }
}

/* ------------------------------------------------------- sum and dot (R8) */

/* One leaf: acc = (+0,+0); for each element, acc = ATF1(acc, term) where
 * the term is x_i (ATF1.1 when x is dotted) for a sum, or the twofold
 * product of x_i and y_i (R6 kinds) for a dot. */
static tfo_tf leaf_reduce(const double *xh, const double *xl, const double *yh,
                          const double *yl, int64_t b, int64_t e, int is_dot) {
    tfo_tf acc = {0.0, 0.0};
    for (int64_t i = b; i < e; ++i) {
        if (!is_dot) {
            if (xl) acc = tfo_atf1(acc.z0, acc.z1, xh[i], xl[i]);
            else    acc = tfo_atf11(acc.z0, acc.z1, xh[i]);
        } else {
            tfo_tf p = op_kinds(TFO_MUL, xh[i], xl ? xl[i] : 0.0, xl == NULL,
                                yh[i], yl ? yl[i] : 0.0, yl == NULL);
            acc = tfo_atf1(acc.z0, acc.z1, p.z0, p.z1);
        }
    }
    return acc;
}

/* Bottom-up pairwise tree in place over nodes[0..m-1]; returns the root. */
static tfo_tf tree_reduce(tfo_tf *nodes, int64_t m) {
    if (m == 0) { tfo_tf z = {0.0, 0.0}; return z; }
    while (m > 1) {
        int64_t h = 0;
        for (int64_t i = 0; i + 1 < m; i += 2)
            nodes[h++] = tfo_atf1(nodes[i].z0, nodes[i].z1, nodes[i + 1].z0, nodes[i + 1].z1);
        if (m & 1) nodes[h++] = nodes[m - 1];
        m = h;
    }
    return nodes[0];
}

/* Twofold sum (is_dot = 0) or dot (is_dot = 1) of n elements with leaf size L.
 * `work` must hold ceil(n/L) twofolds.  Leaf results are also written to
 * `leaves` (if not NULL) so tests can check the tree by parts. */
void tfo_reduce(const double *xh, const double *xl, const double *yh, const double *yl,
                int64_t n, int64_t L, int is_dot, tfo_tf *work, double *z0, double *z1) {
    int64_t m = (n + L - 1) / L;
    for (int64_t j = 0; j < m; ++j) {
        int64_t b = j * L, e = (b + L < n) ? b + L : n;
        work[j] = leaf_reduce(xh, xl, yh, yl, b, e, is_dot);
    }
    tfo_tf r = tree_reduce(work, m);
    *z0 = r.z0;
    *z1 = r.z1;
}

/* Leaf results only (for tests of the tree split and for parallel callers). */
void tfo_reduce_leaves(const double *xh, const double *xl, const double *yh, const double *yl,
                       int64_t n, int64_t L, int is_dot, int64_t j0, int64_t j1, tfo_tf *out) {
    for (int64_t j = j0; j < j1; ++j) {
        int64_t b = j * L, e = (b + L < n) ? b + L : n;
        out[j - j0] = leaf_reduce(xh, xl, yh, yl, b, e, is_dot);
    }
}

/* The tree alone over m given nodes (overwritten). */
void tfo_tree(tfo_tf *nodes, int64_t m, double *z0, double *z1) {
    tfo_tf r = tree_reduce(nodes, m);
    *z0 = r.z0;
    *z1 = r.z1;
}

/* Plain binary64 twin: the same leaves and tree with s = +0; s = s + x_i
 * (sum) or s = s + x_i*y_i (dot, separate multiply and add, no FMA). */
double tfo_reduce_plain(const double *x, const double *y, int64_t n, int64_t L, int is_dot,
                        double *work) {
    int64_t m = (n + L - 1) / L;
    if (m == 0) return 0.0;
    for (int64_t j = 0; j < m; ++j) {
        int64_t b = j * L, e = (b + L < n) ? b + L : n;
        double s = 0.0;
        for (int64_t i = b; i < e; ++i) {
            if (is_dot) { double p = x[i] * y[i]; s = s + p; }
            else        s = s + x[i];
        }
        work[j] = s;
    }
    while (m > 1) {
        int64_t h = 0;
        for (int64_t i = 0; i + 1 < m; i += 2) work[h++] = work[i] + work[i + 1];
        if (m & 1) work[h++] = work[m - 1];
        m = h;
    }
    return work[0];
}

/* ---------------------------------------------------------------- Horner
 * p(x) = a_0 + a_1 x + ... + a_k x^k, coefficients ascending and dotted.
 * s = (a_k, +0); for i = k-1 .. 0: s = ATF1.1(MTF1.1(s, x), a_i). */
void tfo_horner(const double *a, int k, const double *x, int64_t i0, int64_t i1,
                double *out_hi, double *out_lo, unsigned char *flags,
                int mode, double tau, double m) {
    for (int64_t p = i0; p < i1; ++p) {
        tfo_tf s = {a[k], 0.0};
        for (int i = k - 1; i >= 0; --i) {
            tfo_tf t = tfo_mtf11(s.z0, s.z1, x[p]);
            s = tfo_atf11(t.z0, t.z1, a[i]);
        }
        out_hi[p] = s.z0;
        out_lo[p] = s.z1;
        if (flags) flags[p] = tfo_flag(s.z0, s.z1, mode, tau, m);
    }
}

/* Plain twin: s = a_k; s = s*x + a_i with a separate multiply and add. */
void tfo_horner_plain(const double *a, int k, const double *x, int64_t i0, int64_t i1,
                      double *out) {
    for (int64_t p = i0; p < i1; ++p) {
        double s = a[k];
        for (int i = k - 1; i >= 0; --i) {
            double t = s * x[p];
            s = t + a[i];
        }
        out[p] = s;
    }
}
