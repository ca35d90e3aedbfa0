// The leaf level of the blocked pairwise reduction order: one leaf of a
// twofold sum or dot walked left to right,
//   acc = (+0, +0);  acc = ATF1(acc, term_i)  for each element i,
// term_i = x_i for a sum (ATF1.1 when x is dotted: Add/subtract, 2x section)
// and the product of x_i and y_i by the operand kinds for a dot
// (Two-Product, MTF1.1 or MTF1, then ATF1).  The walk is specialised on
// whether x and y are dotted, so no per-element dispatch remains; when the
// leaf's arrays all start on a 16-byte boundary it reads 16-byte pairs, four
// elements per step, and the ragged end one element at a time.  The order
// of the operations is the same either way.
#pragma once
#include "tf_device.cuh"

namespace tf {

// Four consecutive doubles from a 16-byte aligned address, as two 16-byte loads.
__device__ __forceinline__ void ld4(const double *p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// acc = ATF1(acc, term) for one element (x1, y1 are +0 for dotted operands).
// FP: the accumulation's Two-Sum tail by Fast-Two-Sum on ordered operands
// (atf1_fp, same bits).  The dotted dot's step is bound by its integer
// instructions (Two-Product and the Two-Sum tail, ~145 per element against
// 3 FP64 ones), so one element in four takes that form, which balances the
// two pipes; every other kind is bound by its FP64 instructions and keeps
// the integer tail.
template <bool DOT, bool XD, bool YD, bool FP = false>
__device__ __forceinline__ void leaf_term(d2 &acc, double x0, double x1, double y0, double y1) {
    if constexpr (!DOT) {
        acc = XD ? atf11(acc.z0, acc.z1, x0) : atf1(acc.z0, acc.z1, x0, x1);
    } else {
        const d2 p = apply(OP_MUL, x0, x1, XD, y0, y1, YD);
        acc = FP ? atf1_fp(acc.z0, acc.z1, p.z0, p.z1) : atf1(acc.z0, acc.z1, p.z0, p.z1);
    }
}

// The twofold partial of a leaf of len elements starting at X (and XL, Y,
// YL: x tails, y, y tails; the ones the kinds do not use are ignored).
template <bool DOT, bool XD, bool YD>
__device__ __forceinline__ d2 leaf_walk(const double *X, const double *XL, const double *Y, const double *YL,
                                        int64_t len) {
    d2 acc = {0.0, 0.0};
    int64_t i = 0;
    uintptr_t addr = reinterpret_cast<uintptr_t>(X);
    if (!XD) addr |= reinterpret_cast<uintptr_t>(XL);
    if (DOT) addr |= reinterpret_cast<uintptr_t>(Y);
    if (DOT && !YD) addr |= reinterpret_cast<uintptr_t>(YL);
    if ((addr & 15) == 0) {
        for (; i + 4 <= len; i += 4) {
            double x[4], xl[4] = {0.0, 0.0, 0.0, 0.0}, y[4] = {0.0, 0.0, 0.0, 0.0}, yl[4] = {0.0, 0.0, 0.0, 0.0};
            ld4(X + i, x);
            if (!XD) ld4(XL + i, xl);
            if (DOT) ld4(Y + i, y);
            if (DOT && !YD) ld4(YL + i, yl);
#pragma unroll
            for (int u = 0; u < 3; ++u) leaf_term<DOT, XD, YD>(acc, x[u], xl[u], y[u], yl[u]);
            leaf_term<DOT, XD, YD, DOT && XD && YD>(acc, x[3], xl[3], y[3], yl[3]);
        }
    }
    for (; i < len; ++i)
        leaf_term<DOT, XD, YD>(acc, X[i], XD ? 0.0 : XL[i], DOT ? Y[i] : 0.0, (DOT && !YD) ? YL[i] : 0.0);
    return acc;
}

}  // namespace tf
