/*
 * Seeded synthetic input generators for the twofold workloads.
 *
 * This module produces INPUTS only.  It holds none of the twofold method's
 * arithmetic (no Two-Sum, Two-Product, ATF/MTF/DTF/RTF step): both the CPU
 * oracle and the CUDA library consume what it writes, and neither is linked
 * into it.  The one piece of arithmetic beyond plain sampling is an exact
 * (Kulisch-style, pure integer) dot-product accumulator, used to construct
 * ill-conditioned dot products and to report their exact value.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator: output i of stream k under seed s is
 *     mix64(key(s,k) + (i+1) * 0x9E3779B97F4A7C15),  key(s,k) = mix64(s + (k+1) * 0xD1B54A32D192ED03)
 * so any index range can be produced independently (and in parallel).
 *
 * Build: plain C99, no contraction of floating-point expressions
 * (-ffp-contract=off), so x86_64 and aarch64 hosts write identical bits.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <math.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL
#define STREAM_GAP 0xD1B54A32D192ED03ULL

static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return mix64(seed + (stream + 1) * STREAM_GAP);
}

/* i-th 64-bit output of (seed, stream). */
uint64_t synth_u64(uint64_t seed, uint64_t stream, uint64_t i) {
    return mix64(stream_key(seed, stream) + (i + 1) * GOLDEN);
}

/* 53-bit uniform in [0, 1): top 53 bits of the word times 2^-53 (exact). */
static double u01(uint64_t w) { return (double)(w >> 11) * 0x1p-53; }

/* ulp of a finite double: 2^(max(e,-1022)-52); ulp(0) = 2^-1074. */
static double ulp_of(double h) {
    uint64_t b;
    memcpy(&b, &h, 8);
    int e = (int)((b >> 52) & 0x7FF);
    if (e == 0) e = 1;               /* subnormal or zero: spacing 2^-1074 */
    return ldexp(1.0, e - 1023 - 52);
}

/* out[j] = lo + (hi - lo) * U_{i0+j}, U uniform on [0,1). */
void synth_uniform(uint64_t seed, uint64_t stream, int64_t i0, int64_t n,
                   double lo, double hi, double *out) {
    uint64_t key = stream_key(seed, stream);
    double w = hi - lo;
    for (int64_t j = 0; j < n; ++j) {
        uint64_t r = mix64(key + (uint64_t)(i0 + j + 1) * GOLDEN);
        double t = w * u01(r);
        out[j] = lo + t;
    }
}

/* Log-uniform magnitudes 10^(e_lo + (e_hi - e_lo) U); when `signed_` is set
 * the sign is the lowest bit of the same word (bits 11..63 feed U). */
void synth_loguniform(uint64_t seed, uint64_t stream, int64_t i0, int64_t n,
                      double e_lo, double e_hi, int signed_, double *out) {
    uint64_t key = stream_key(seed, stream);
    const double ln10 = 2.302585092994045684;
    double w = e_hi - e_lo;
    for (int64_t j = 0; j < n; ++j) {
        uint64_t r = mix64(key + (uint64_t)(i0 + j + 1) * GOLDEN);
        double t = w * u01(r);
        double e = e_lo + t;
        double m = exp(e * ln10);
        out[j] = (signed_ && (r & 1)) ? -m : m;
    }
}

/* Tails uniform in [-1/2, 1/2) ulp of the matching head: (U - 1/2) * ulp(h),
 * exact because ulp(h) is a power of two (heads are in the normal range). */
void synth_ulp_tails(uint64_t seed, uint64_t stream, int64_t i0, int64_t n,
                     const double *heads, double *out) {
    uint64_t key = stream_key(seed, stream);
    for (int64_t j = 0; j < n; ++j) {
        uint64_t r = mix64(key + (uint64_t)(i0 + j + 1) * GOLDEN);
        double c = u01(r) - 0.5;
        out[j] = c * ulp_of(heads[j]);
    }
}

/* ------------------------------------------------------------------------
 * Exact dot-product accumulator (pure integer).
 *
 * A finite double is m * 2^q with integer |m| < 2^53 and q >= -1074, so a
 * product of two is M * 2^Q with |M| < 2^106 and Q >= -2148.  The sum is
 * kept as a two's-complement integer N with value N * 2^-2148, in NLIMB
 * 64-bit limbs: 2^(2048+64) covers products up to the overflow threshold
 * with 64 bits of headroom for the count of terms.
 * ---------------------------------------------------------------------- */
#define ACC_BIAS 2148
#define NLIMB 68

typedef struct { uint64_t w[NLIMB]; } xacc;

static void acc_clear(xacc *a) { memset(a, 0, sizeof(*a)); }

/* decompose finite x = m * 2^q, m signed 54-bit integer */
static void decomp(double x, int64_t *m, int *q) {
    uint64_t b;
    memcpy(&b, &x, 8);
    int e = (int)((b >> 52) & 0x7FF);
    uint64_t f = b & 0xFFFFFFFFFFFFFULL;
    if (e == 0) { *q = -1074; } else { f |= 1ULL << 52; *q = e - 1075; }
    *m = (b >> 63) ? -(int64_t)f : (int64_t)f;
}

/* add (neg ? -1 : +1) * v * 2^pos, v < 2^128, to the accumulator */
static void acc_add_shifted(xacc *a, unsigned __int128 v, int pos, int neg) {
    if (v == 0) return;
    int li = pos >> 6, sh = pos & 63;
    uint64_t p[3];
    p[0] = (uint64_t)v << sh;
    p[1] = sh ? (uint64_t)(v >> (64 - sh)) : (uint64_t)(v >> 64);
    p[2] = sh ? (uint64_t)(v >> (128 - sh)) : 0;
    if (!neg) {
        uint64_t carry = 0;
        for (int k = 0; li + k < NLIMB; ++k) {
            uint64_t add = (k < 3) ? p[k] : 0;
            if (k >= 3 && carry == 0) break;
            uint64_t s = a->w[li + k] + add;
            uint64_t c1 = s < add;
            uint64_t s2 = s + carry;
            uint64_t c2 = s2 < carry;
            a->w[li + k] = s2;
            carry = c1 | c2;
        }
    } else {
        uint64_t borrow = 0;
        for (int k = 0; li + k < NLIMB; ++k) {
            uint64_t sub = (k < 3) ? p[k] : 0;
            if (k >= 3 && borrow == 0) break;
            uint64_t old = a->w[li + k];
            uint64_t d = old - sub;
            uint64_t b1 = old < sub;
            uint64_t d2 = d - borrow;
            uint64_t b2 = d < borrow;
            a->w[li + k] = d2;
            borrow = b1 | b2;
        }
    }
}

static void acc_add_prod(xacc *a, double x, double y) {
    int64_t mx, my; int qx, qy;
    decomp(x, &mx, &qx);
    decomp(y, &my, &qy);
    if (mx == 0 || my == 0) return;
    int neg = (mx < 0) ^ (my < 0);
    unsigned __int128 v = (unsigned __int128)(uint64_t)(mx < 0 ? -mx : mx) *
                          (unsigned __int128)(uint64_t)(my < 0 ? -my : my);
    acc_add_shifted(a, v, qx + qy + ACC_BIAS, neg);
}

/* Round the accumulator to the nearest double (ties to even). */
static double acc_round(const xacc *a) {
    xacc m = *a;
    int neg = (int)(m.w[NLIMB - 1] >> 63);
    if (neg) {  /* two's-complement negate */
        uint64_t carry = 1;
        for (int k = 0; k < NLIMB; ++k) {
            uint64_t v = ~m.w[k] + carry;
            carry = (carry && v == 0);
            m.w[k] = v;
        }
    }
    int top = -1;
    for (int k = NLIMB - 1; k >= 0; --k)
        if (m.w[k]) { top = k * 64 + 63 - __builtin_clzll(m.w[k]); break; }
    if (top < 0) return 0.0;
    /* value = M * 2^-ACC_BIAS, leading bit at `top`; keep bits down to `lo` */
    int lead_exp = top - ACC_BIAS;
    int lo = (lead_exp >= -1022) ? top - 52 : (-1074 + ACC_BIAS);
    if (lo < 0) lo = 0;
    uint64_t mant = 0;
    for (int bit = top; bit >= lo; --bit)
        mant = (mant << 1) | ((m.w[bit >> 6] >> (bit & 63)) & 1);
    int round = 0, sticky = 0;
    if (lo > 0) {
        int rb = lo - 1;
        round = (int)((m.w[rb >> 6] >> (rb & 63)) & 1);
        for (int bit = rb - 1; bit >= 0 && !sticky; --bit) {
            if ((bit & 63) == 63 && m.w[bit >> 6] == 0) { bit -= 63; continue; }
            sticky |= (int)((m.w[bit >> 6] >> (bit & 63)) & 1);
        }
    }
    if (round && (sticky || (mant & 1))) mant += 1;
    double r = ldexp((double)mant, lo - ACC_BIAS);
    return neg ? -r : r;
}

/* Exact dot of x and y rounded to nearest (*dot_rn), and the condition
 * number 2 * sum|x_i y_i| / |sum x_i y_i| (*cond), both from exact sums. */
void synth_exact_dot(const double *x, const double *y, int64_t n,
                     double *dot_rn, double *cond) {
    static __thread xacc s, sa;
    acc_clear(&s); acc_clear(&sa);
    for (int64_t i = 0; i < n; ++i) {
        acc_add_prod(&s, x[i], y[i]);
        acc_add_prod(&sa, fabs(x[i]), fabs(y[i]));
    }
    double d = acc_round(&s), m = acc_round(&sa);
    *dot_rn = d;
    *cond = (d == 0.0) ? INFINITY : 2.0 * m / fabs(d);
}

/* Exact sum of x (plus optional tails xl) rounded to nearest. */
double synth_exact_sum(const double *x, const double *xl, int64_t n) {
    static __thread xacc s;
    acc_clear(&s);
    for (int64_t i = 0; i < n; ++i) {
        acc_add_prod(&s, x[i], 1.0);
        if (xl) acc_add_prod(&s, xl[i], 1.0);
    }
    return acc_round(&s);
}

/* ------------------------------------------------------------------------
 * Ill-conditioned dot product of length n (n >= 6) with target condition
 * `cond`, after the construction idea of Ogita, Rump and Oishi ("Accurate
 * sum and dot product", SIAM J. Sci. Comput. 26(6), 2005, Sect. 6), written
 * from that description with an exact accumulator in place of their
 * compensated running dot:
 *   - b = log2(cond); the first n - m pairs get random mantissas in [-1,1)
 *     and exponents drawn from [0, b/2] (the first forced to b/2, the last
 *     to 0); m = min(n/2, 32) (the published construction cancels over
 *     n/2 pairs, which cannot reach conditions below about n; a short tail
 *     reaches down to about 2m),
 *   - the last m pairs get exponents moving linearly from b/2 to e_f and
 *     y_i = (r_i * 2^e_i - D) / x_i, D = nearest double to the exact running
 *     dot, so the running dot follows r_i * 2^e_i and ends near 2^e_f,
 *   - e_f starts at log2(4 S1 / cond), S1 = sum |x_i y_i| of the first part,
 *     and is corrected by log2(realised / target) for up to 4 passes (the
 *     random draws are the same in every pass; only exponents move),
 *   - the pairs are then shuffled (Fisher-Yates, same RNG).
 * The exact dot and the realised condition number are returned.
 * ---------------------------------------------------------------------- */
static void cond_dot_pass(uint64_t seed, int64_t n, double bh, double ef,
                          double *x, double *y, double *s1_out) {
    static __thread xacc s;
    uint64_t kx = stream_key(seed, 0), ky = stream_key(seed, 1);
    uint64_t ke = stream_key(seed, 2);
    int64_t n2 = n - ((n / 2 < 32) ? n / 2 : 32);
    double s1 = 0.0;
    acc_clear(&s);
    for (int64_t i = 0; i < n2; ++i) {
        double re = u01(mix64(ke + (uint64_t)(i + 1) * GOLDEN));
        int e = (int)floor(re * (bh + 1.0));
        if (i == 0) e = (int)floor(bh + 0.5) + 1;
        if (i == n2 - 1) e = 0;
        double rx = 2.0 * u01(mix64(kx + (uint64_t)(i + 1) * GOLDEN)) - 1.0;
        double ry = 2.0 * u01(mix64(ky + (uint64_t)(i + 1) * GOLDEN)) - 1.0;
        x[i] = ldexp(rx, e);
        y[i] = ldexp(ry, e);
        s1 += fabs(x[i] * y[i]);
        acc_add_prod(&s, x[i], y[i]);
    }
    for (int64_t i = n2; i < n; ++i) {
        double frac = (n - 1 == n2) ? 0.0 : (double)(n - 1 - i) / (double)(n - 1 - n2);
        int e = (int)floor(ef + (bh - ef) * frac + 0.5);
        double rx = 2.0 * u01(mix64(kx + (uint64_t)(i + 1) * GOLDEN)) - 1.0;
        double ry = 2.0 * u01(mix64(ky + (uint64_t)(i + 1) * GOLDEN)) - 1.0;
        if (rx == 0.0) rx = 0.5;
        if (ry == 0.0) ry = 0.5;
        x[i] = ldexp(rx, e);
        double d = acc_round(&s);
        double num = ldexp(ry, e) - d;
        y[i] = num / x[i];
        acc_add_prod(&s, x[i], y[i]);
    }
    *s1_out = s1;
}

void synth_cond_dot(uint64_t seed, int64_t n, double cond, double *x, double *y,
                    double *dot_rn, double *cond_out) {
    uint64_t kp = stream_key(seed, 3);
    double bh = 0.5 * log2(cond);
    double s1 = 0.0, d = 0.0, c = 0.0;
    cond_dot_pass(seed, n, bh, 0.0, x, y, &s1);
    double ef = log2(4.0 * s1 / cond);
    for (int pass = 0; pass < 4; ++pass) {
        cond_dot_pass(seed, n, bh, ef, x, y, &s1);
        synth_exact_dot(x, y, n, &d, &c);
        double adj = log2(c / cond);
        if (!(fabs(adj) > 0.5) || !isfinite(adj)) break;
        ef += adj;
    }
    for (int64_t i = n - 1; i > 0; --i) {
        uint64_t r = mix64(kp + (uint64_t)(i + 1) * GOLDEN);
        int64_t j = (int64_t)(r % (uint64_t)(i + 1));
        double tx = x[i]; x[i] = x[j]; x[j] = tx;
        double ty = y[i]; y[i] = y[j]; y[j] = ty;
    }
    synth_exact_dot(x, y, n, dot_rn, cond_out);
}
